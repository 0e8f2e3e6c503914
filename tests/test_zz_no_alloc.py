"""The allocation-free right-hand side, lor_rhs_static, against lor_rhs.

Callers that may not call cudaMalloc (their framework owns all device memory,
or their device-memory budget is fixed at start-up) cannot build a solver
context; lor_rhs_static serves them with its scratch in a static device array.
This file runs after the context-based tests (ordered in conftest.py): it checks,
through the C ABI, that two calls in a row give the same b as the context-based
entry point, within the 1e-12 relative tolerance the right-hand-side parity test
uses, and that sizes beyond the static array are refused.
"""
import ctypes

import numpy as np
import pytest

from paper_1908_07071_gb300.synthetic import make_mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1908_07071_gb300.build import build_library
    build_library()


@pytest.mark.parametrize("dim,n,p", [(2, 8, 4), (3, (3, 4, 5), 3), (3, 6, 8)])
def test_rhs_static_matches_rhs(dim, n, p):
    from paper_1908_07071_gb300 import lor
    lib = lor.load()
    verts, kappa = make_mesh(dim, n, seed=2, perturb=0.15)
    s = lor.Solver(verts, kappa, p)
    nn = list(reversed(kappa.shape)) + [1]
    dv = torch.from_numpy(np.ascontiguousarray(verts).ravel()).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for kind in (0, 1):
        ref = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
        s.rhs(ref, kind)
        for _ in range(2):                     # two calls in a row share the static scratch
            b = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
            st = lib.lor_rhs_static(dim, p, nn[0], nn[1], nn[2], ctypes.c_void_p(dv.data_ptr()), kind,
                                    ctypes.c_void_p(b.data_ptr()), stream)
            assert st == lor.LOR_OK
            torch.cuda.synchronize()
            r = ref.cpu().numpy()
            assert np.abs(b.cpu().numpy() - r).max() <= 1e-12 * np.abs(r).max()
    s.close()


def test_rhs_static_rejects_oversize():
    from paper_1908_07071_gb300 import lor
    lib = lor.load()
    dv = torch.zeros(3 * 17 ** 3, dtype=torch.float64, device="cuda")
    b = torch.zeros(8, dtype=torch.float64, device="cuda")
    # 16^3 elements x 9^3 points = 2,985,984 > 2^21 - 256 doubles of static scratch
    st = lib.lor_rhs_static(3, 8, 16, 16, 16, ctypes.c_void_p(dv.data_ptr()), 0, ctypes.c_void_p(b.data_ptr()),
                            None)
    assert st == lor.LOR_EINVAL
    assert lib.lor_rhs_static(3, 9, 2, 2, 2, ctypes.c_void_p(dv.data_ptr()), 0, ctypes.c_void_p(b.data_ptr()),
                              None) == lor.LOR_EINVAL
