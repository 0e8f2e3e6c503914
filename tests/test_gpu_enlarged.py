"""Patches enlarged for isotropic overlap on the GPU (lor_set_patch_spans; Section 4.5):
on anisotropic strip meshes every vertex patch takes whole elements across the thin
strip until its overlap is isotropic (the oracle's isotropic_overlap_spans), the
element-structured V(1,1) cycle runs on the enlarged boxes, and a box that keeps
several vertices on its coarsest level solves them exactly.  B r in FP64 equals the
oracle's LORPreconditioner(patch_spans=...) to 1e-10 relative (max-norm), FP32 stays
within the bounds of the vertex-patch FP32 test, and PCG counts are within one
iteration of the oracle's; the count stays flat in the aspect ratio."""
import numpy as np
import pytest

from oracle import cg, krylov
from oracle import lor as olor
from oracle.mesh import Mesh
from paper_1908_07071_gb300.synthetic import make_mesh, make_strip_mesh, random_vector

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
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _span_array(spans, n, dim):
    """Oracle spans {vertex: [(lo, hi) per axis]} as the library's (npatch, dim, 2) array."""
    shape = [v + 1 for v in n]
    J = int(np.prod(shape))
    out = np.ones((J, dim, 2), dtype=np.int32)
    for v, per in spans.items():
        j = v[0] + shape[0] * (v[1] + (shape[1] * v[2] if dim == 3 else 0))
        out[j] = np.array(per, dtype=np.int32)
    return out


def _check_apply(v, k, p, spans, mg=0):
    from paper_1908_07071_gb300 import lor
    m = Mesh(v, k)
    B = olor.LORPreconditioner(m, p, mg_levels=mg, patch_spans=spans)
    arr = _span_array(spans, m.n, m.dim)
    r = random_vector(int(np.prod([x * p + 1 for x in m.n])), 41)
    z_ref = B.apply(r)
    for bf16 in (False, True):
        s = lor.Solver(v, k, p, mg_levels=mg, patch_spans=arr, factor_bf16=bf16)
        if not bf16:
            z = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
            s.apply_P(torch.from_numpy(r).cuda(), z)
            assert _rel(z.cpu().numpy(), z_ref) < 1e-10
        z32 = torch.empty(s.nvec, dtype=torch.float32, device="cuda")
        s.apply_P(torch.from_numpy(r).float().cuda(), z32, prec=lor.LOR_FP32)
        err = _rel(z32.double().cpu().numpy(), z_ref)
        assert err < (8 * 2.0 ** -8 if bf16 else 50 * U32 * 1e3), err
        s.close()
    return B


@pytest.mark.parametrize("p,aspect", [(3, 15.0), (3, 150.0), (2, 1500.0), (5, 15.0), (1, 150.0)])
def test_strip_mesh_enlarged_patches_match_oracle(p, aspect):
    v, k = make_strip_mesh(8, aspect, layers=4, seed=0)
    spans = olor.isotropic_overlap_spans(Mesh(v, k))
    assert max(max(max(t) for t in per) for per in spans.values()) > 1   # some patches are enlarged
    _check_apply(v, k, p, spans)


def test_3d_enlarged_patches_match_oracle():
    """3D boxes spanning up to three elements along an axis, with several vertices on
    their coarsest level, on a perturbed mesh (spans chosen by hand, seeded)."""
    v, k = make_mesh(3, (3, 4, 3), seed=7, perturb=0.15)
    m = Mesh(v, k)
    rng = np.random.default_rng(3)
    spans = {}
    for z in range(m.n[2] + 1):
        for y in range(m.n[1] + 1):
            for x in range(m.n[0] + 1):
                spans[(x, y, z)] = [tuple(int(t) for t in rng.integers(1, 3, 2)) for _ in range(3)]
    _check_apply(v, k, 3, spans)
    _check_apply(v, k, 4, spans, mg=2)


@pytest.mark.parametrize("aspect", [1.5, 150.0])
def test_enlarged_pcg_matches_oracle(aspect):
    from paper_1908_07071_gb300 import lor
    v, k = make_strip_mesh(8, aspect, layers=4, seed=0)
    m = Mesh(v, k)
    p = 3
    spans = olor.isotropic_overlap_spans(m)
    rtol = 1e-10
    K = cg.assemble_stiffness(m, p)
    N = cg.node_shape(m.n, p)
    B = olor.LORPreconditioner(m, p, patch_spans=spans)
    b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
    _, it_or, _, _ = krylov.pcg(lambda u: cg.apply_A(K, N, u), B.apply, b, rtol=rtol)
    s = lor.Solver(v, k, p, rtol=rtol, patch_spans=_span_array(spans, m.n, m.dim))
    x = torch.zeros(s.nvec, dtype=torch.float64, device="cuda")
    it, rel = s.solve(torch.from_numpy(b).cuda(), x)
    print(f"enlarged patches, aspect {aspect}: GPU {it}, oracle {it_or}")
    assert abs(it - it_or) <= 1 and rel <= rtol
    s.close()


def test_patch_spans_are_checked():
    from paper_1908_07071_gb300 import lor
    v, k = make_mesh(2, 3, seed=7, perturb=0.15)
    bad = np.ones((16, 2, 2), dtype=np.int32)
    bad[5, 1, 0] = 0
    with pytest.raises(lor.LorError) as err:
        lor.Solver(v, k, 2, patch_spans=bad)
    assert err.value.status == lor.LOR_EINVAL
    with pytest.raises(ValueError):
        lor.Solver(v, k, 2, patch_spans=np.ones((15, 2, 2), dtype=np.int32))
    s = lor.Solver(v, k, 2, patch_spans=np.ones((16, 2, 2), dtype=np.int32))
    with pytest.raises(lor.LorError) as err:
        s.set_weighting(1)
    assert err.value.status == lor.LOR_EINVAL
    s.close()
