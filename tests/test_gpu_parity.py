"""GPU-vs-oracle parity of the CG path through the C ABI (needs a GB300).

Tolerances: FP64 results agree with the FP64 oracle to 1e-10 relative (max-norm
over the vector); FP32 results obey the componentwise bound
|y32 - y| <= c u32 (|A| |x|) with u32 = 2^-24 and c stated per test; solves are
compared with the oracle's own iteration counts (+-1) and with a direct solve.
"""
import numpy as np
import pytest

from oracle import cg, krylov
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


def _solver(verts, kappa, p, **kw):
    from paper_1908_07071_gb300 import lor
    return lor.Solver(verts, kappa, p, **kw)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = [  # (dim, n, p, perturb, kappa_const, mg_levels)
    (2, 8, 4, 0.0, 1.0, 2),       # the 2D Q4 8x8 manufactured problem
    (2, 5, 3, 0.15, None, 0),
    (2, (3, 4), 6, 0.15, None, 0),  # ragged: nx != ny
    (3, 3, 2, 0.15, None, 0),
    (3, 3, 4, 0.15, None, 0),
    (3, (2, 3, 4), 3, 0.15, None, 0),
    (3, 2, 8, 0.15, None, 0),
    (3, 2, 6, 0.15, None, 2),
    (3, 1, 3, 0.15, None, 0),     # single element: no interior vertex
    (3, 3, 1, 0.15, None, 0),     # p = 1: the patch box is the vertex level (one unknown)
    (2, 4, 1, 0.15, None, 0),
]


def _problem(dim, n, p, pert, kc, mg, seed=0):
    verts, kappa = make_mesh(dim, n, seed=seed, perturb=pert, kappa_const=kc)
    return verts, kappa, Mesh(verts, kappa)


@pytest.mark.parametrize("case", CASES, ids=str)
def test_apply_A_fp64_and_fp32(case):
    from paper_1908_07071_gb300 import lor
    dim, n, p, pert, kc, mg = case
    verts, kappa, m = _problem(*case)
    s = _solver(verts, kappa, p, mg_levels=mg)
    K = cg.assemble_stiffness(m, p)
    N = cg.node_shape(m.n, p)
    x = random_vector(s.nvec, 11)
    y_ref = cg.apply_A(K, N, x)
    xd = torch.from_numpy(x).cuda()
    y = torch.full_like(xd, np.nan)
    s.apply_A(xd, y)
    assert _rel(y.cpu().numpy(), y_ref) < 1e-10
    # FP32: |y32 - y| <= 64 u32 (|K| |x|) componentwise (sum-factorized rounding)
    y32 = torch.empty(s.nvec, dtype=torch.float32, device="cuda")
    s.apply_A(xd.float(), y32, prec=lor.LOR_FP32)
    bound = 64 * U32 * cg.apply_A(abs(K), N, np.abs(x)) + 1e-30
    assert np.all(np.abs(y32.double().cpu().numpy() - y_ref) <= bound)
    s.close()


@pytest.mark.parametrize("case", CASES, ids=str)
def test_apply_P_fp64(case):
    dim, n, p, pert, kc, mg = case
    verts, kappa, m = _problem(*case)
    s = _solver(verts, kappa, p, mg_levels=mg)
    B = olor.LORPreconditioner(m, p, mg_levels=mg)
    r = random_vector(s.nvec, 12)
    z_ref = B.apply(r)
    z = torch.full((s.nvec,), np.nan, dtype=torch.float64, device="cuda")
    s.apply_P(torch.from_numpy(r).cuda(), z)
    assert _rel(z.cpu().numpy(), z_ref) < 1e-10
    s.close()


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("case", [CASES[0], CASES[4], CASES[6]], ids=str)
def test_apply_P_fp32(case, bf16):
    """FP32 preconditioner: fp32 stencils, fp32 or bf16 ILU factors.  Bound: the
    relative max-norm error stays below 50 u32 * kappa_P (fp32 factors) or 8 u_bf16
    (bf16 factors), with kappa_P ~ 1e3 the amplification of one V-cycle."""
    from paper_1908_07071_gb300 import lor
    dim, n, p, pert, kc, mg = case
    verts, kappa, m = _problem(*case)
    s = _solver(verts, kappa, p, mg_levels=mg, factor_bf16=bf16)
    B = olor.LORPreconditioner(m, p, mg_levels=mg)
    r = random_vector(s.nvec, 13)
    z_ref = B.apply(r)
    z = torch.empty(s.nvec, dtype=torch.float32, device="cuda")
    s.apply_P(torch.from_numpy(r).float().cuda(), z, prec=lor.LOR_FP32)
    err = _rel(z.double().cpu().numpy(), z_ref)
    assert err < (8 * 2.0 ** -8 if bf16 else 50 * U32 * 1e3), err
    s.close()


def test_mesh_from_device_arrays():
    """lor_create reads vertices and kappa from device memory as well as from host memory: a
    context built from torch CUDA tensors applies A and B like the oracle (1e-10) and bit for bit
    like the context built from the same arrays on the host."""
    verts, kappa, m = _problem(3, (3, 2, 2), 4, 0.15, None, 0)
    s_dev = _solver(torch.from_numpy(verts).cuda(), torch.from_numpy(kappa).cuda(), 4)
    s_host = _solver(verts, kappa, 4)
    x = torch.from_numpy(random_vector(s_dev.nvec, 14)).cuda()
    y_dev, y_host = torch.empty_like(x), torch.empty_like(x)
    s_dev.apply_A(x, y_dev)
    s_host.apply_A(x, y_host)
    assert torch.equal(y_dev, y_host)
    N = cg.node_shape(m.n, 4)
    assert _rel(y_dev.cpu().numpy(), cg.apply_A(cg.assemble_stiffness(m, 4), N, x.cpu().numpy())) < 1e-10
    s_dev.apply_P(x, y_dev)
    s_host.apply_P(x, y_host)
    assert torch.equal(y_dev, y_host)
    assert _rel(y_dev.cpu().numpy(), olor.LORPreconditioner(m, 4).apply(x.cpu().numpy())) < 1e-10
    s_dev.close()
    s_host.close()


def test_rhs_matches_oracle_load_vector():
    for dim, n, p in ((2, 4, 3), (3, 2, 4)):
        verts, kappa = make_mesh(dim, n, seed=5, perturb=0.15)
        m = Mesh(verts, kappa)
        s = _solver(verts, kappa, p)
        b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
        for kind, f in ((0, lambda X: np.ones(len(X))),
                        (1, lambda X: dim * np.pi ** 2 * np.prod(np.sin(np.pi * X), axis=1))):
            s.rhs(b, kind)
            ref = cg.load_vector(m, p, f, q=p + 1)
            assert _rel(b.cpu().numpy(), ref) < 1e-12
        s.close()


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[4], CASES[5]], ids=str)
def test_pcg_fp64_matches_oracle(case):
    dim, n, p, pert, kc, mg = case
    verts, kappa, m = _problem(*case)
    rtol = 1e-10
    s = _solver(verts, kappa, p, mg_levels=mg, rtol=rtol)
    K = cg.assemble_stiffness(m, p)
    N = cg.node_shape(m.n, p)
    B = olor.LORPreconditioner(m, p, mg_levels=mg)
    b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
    x_or, it_or, hist_or, coef = krylov.pcg(lambda u: cg.apply_A(K, N, u), B.apply, b, rtol=rtol)
    x = torch.zeros(s.nvec, dtype=torch.float64, device="cuda")
    it, rel = s.solve(torch.from_numpy(b).cuda(), x)
    assert abs(it - it_or) <= 1, (it, it_or)
    assert rel <= rtol
    hist = s.history()
    np.testing.assert_allclose(hist[: min(len(hist), 6)], hist_or[: min(len(hist), 6)], rtol=1e-8)
    lo, hi = krylov.lanczos_condition(*coef)
    kappa_est = hi / lo
    xs = x.cpu().numpy()
    # forward error bound: kappa * (||r_gpu|| + ||r_oracle||) / ||b||
    assert np.linalg.norm(xs - x_or) / np.linalg.norm(x_or) <= kappa_est * 2 * rtol * 10
    s.close()


def test_pcg_host_buffers_and_repeatability():
    verts, kappa, m = _problem(*CASES[4])
    s = _solver(verts, kappa, 4)
    b = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    s.rhs(b, 0)
    x1 = torch.zeros_like(b)
    it1, r1 = s.solve(b, x1)
    hb = b.cpu().numpy().copy()
    hx = np.zeros_like(hb)
    it2, r2 = s.solve_host(hb, hx)
    # scatter-adds use atomics, so repeated solves agree to rounding, not bitwise
    assert abs(it1 - it2) <= 1 and r2 <= 1e-8
    x1h = x1.cpu().numpy()
    assert np.linalg.norm(hx - x1h) <= 1e-9 * np.linalg.norm(x1h)
    s.close()


@pytest.mark.parametrize("bf16", [False, True])
def test_mixed_precision_reaches_fp64_accuracy(bf16):
    from paper_1908_07071_gb300 import lor
    verts, kappa, m = _problem(3, 4, 4, 0.15, None, 0)
    rtol = 1e-8
    s64 = _solver(verts, kappa, 4, rtol=rtol)
    smx = _solver(verts, kappa, 4, rtol=rtol, prec=lor.LOR_MIXED, factor_bf16=bf16)
    b = torch.empty(s64.nvec, dtype=torch.float64, device="cuda")
    s64.rhs(b, 0)
    x64 = torch.zeros_like(b)
    xmx = torch.zeros_like(b)
    it64, r64 = s64.solve(b, x64)
    itmx, rmx = smx.solve(b, xmx)
    assert r64 <= rtol and rmx <= rtol, (r64, rmx)
    hist = smx.history()
    assert hist[-1] / hist[0] <= rtol
    K = cg.assemble_stiffness(m, 4)
    N = cg.node_shape(m.n, 4)
    bo = b.cpu().numpy()
    res = np.linalg.norm(bo - cg.apply_A(K, N, xmx.cpu().numpy())) / np.linalg.norm(bo)
    assert res <= rtol * 1.01      # FP64 residual recomputed by the oracle
    print(f"mixed precision (bf16 factors {bf16}): {itmx} inner iterations, FP64 PCG {it64}")
    # the FP32 preconditioner (fp32 or bf16 factors) perturbs B by 1e-7..1e-2 relative and the
    # refinement restarts the inner flexible CG; measured 80 vs 74 here, 161 vs 152 at Q8 32^3
    assert itmx <= 1.15 * it64 + 2
    s64.close()
    smx.close()


def test_full_size_properties_p8_n32():
    """The 3D p=8, 32^3 workload at full size: sampled operator rows against the
    oracle's element matrices, symmetry of A and B, positivity of B."""
    from paper_1908_07071_gb300 import lor
    verts, kappa = make_mesh(3, 32, seed=0, perturb=0.15)
    m = Mesh(verts, kappa)
    p = 8
    s = _solver(verts, kappa, p)
    x = random_vector(s.nvec, 21)
    y = torch.empty(s.nvec, dtype=torch.float64, device="cuda")
    xd = torch.from_numpy(x).cuda()
    s.apply_A(xd, y)
    rng = np.random.default_rng(0)
    rows = rng.integers(0, s.nvec, 40)
    N = cg.node_shape(m.n, p)
    yo = cg.apply_A_rows(m, p, x, rows)
    yg = y.cpu().numpy()[rows]
    assert np.abs(yg - yo).max() <= 1e-10 * np.abs(yg).max()
    x2 = torch.from_numpy(random_vector(s.nvec, 22)).cuda()
    mask = torch.from_numpy(~cg.boundary_mask(N)).cuda()
    x2 = torch.where(mask, x2, 0)
    xd = torch.where(mask, xd, 0)
    y2 = torch.empty_like(y)
    s.apply_A(x2, y2)
    s.apply_A(xd, y)
    a, b2 = float(x2 @ y), float(xd @ y2)
    assert abs(a - b2) <= 1e-11 * abs(a)
    z = torch.empty_like(y)
    z2 = torch.empty_like(y)
    s.apply_P(xd, z)
    s.apply_P(x2, z2)
    a, b2 = float(x2 @ z), float(xd @ z2)
    assert abs(a - b2) <= 1e-10 * abs(a)
    assert float(xd @ z) > 0 and float(x2 @ z2) > 0
    s.close()


def test_full_size_patch_vcycle_sampled_p8():
    """apply_P at p=8 on a 32^3 mesh with a right-hand side supported on one node:
    z is the sum of the 8 patch V-cycles containing the node plus the coarse term.
    The patch part is checked against an oracle built on the 3x3x3 sub-mesh around
    the node's element (patch matrices only depend on the elements of the patch)."""
    verts, kappa = make_mesh(3, 32, seed=0, perturb=0.15)
    p = 8
    s = _solver(verts, kappa, p)
    e0 = (13, 17, 9)                      # element holding the node
    loc = (3, 5, 2)                       # element-interior GLL position
    Nx = 32 * p + 1
    I = [e0[a] * p + loc[a] for a in range(3)]
    node = (I[2] * Nx + I[1]) * Nx + I[0]
    r = torch.zeros(s.nvec, dtype=torch.float64, device="cuda")
    r[node] = 1.0
    z = torch.empty_like(r)
    s.apply_P(r, z)
    # sub-mesh of elements e0-1 .. e0+1 in each direction
    sub_v = verts[:, e0[2] - 1:e0[2] + 3, e0[1] - 1:e0[1] + 3, e0[0] - 1:e0[0] + 3].copy()
    sub_k = kappa[e0[2] - 1:e0[2] + 2, e0[1] - 1:e0[1] + 2, e0[0] - 1:e0[0] + 2].copy()
    sm = Mesh(sub_v, sub_k)
    corners = [(1 + a, 1 + b, 1 + c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
    B = olor.LORPreconditioner(sm, p, patch_subset=corners, coarse=False)
    Ns = cg.node_shape(sm.n, p)
    rs = np.zeros(int(np.prod(Ns)))
    Il = [p + loc[a] for a in range(3)]
    rs[(Il[2] * Ns[1] + Il[1]) * Ns[0] + Il[0]] = 1.0
    zs = B.apply(rs, parts=("patches",))
    # coarse part: P_0 e with e from the GPU is not separable; compare the sub-box
    # of z that only the 8 patches reach, minus the coarse correction, which is the
    # Q1 interpolant of a vertex vector and therefore exactly trilinear in each
    # element's reference coordinates.  Instead check the patch part directly on
    # nodes where the difference z - zs is trilinear: compare second differences.
    zg = z.cpu().numpy().reshape(Nx, Nx, Nx)
    zsub = zg[e0[2] * p - p:e0[2] * p + 2 * p + 1, e0[1] * p - p:e0[1] * p + 2 * p + 1,
              e0[0] * p - p:e0[0] * p + 2 * p + 1]
    d = zsub - zs.reshape(Ns[2], Ns[1], Ns[0])
    # inside the central element, d = P_0 e is a trilinear function of the GLL
    # reference coordinates: fit it from the 8 corners and compare everywhere
    from oracle.basis import gll
    xg = gll(p)[0]
    ce = d[p:2 * p + 1, p:2 * p + 1, p:2 * p + 1]
    fit = np.zeros_like(ce)
    for c in range(8):
        bx, by, bz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        wx = xg if bx else 1 - xg
        wy = xg if by else 1 - xg
        wz = xg if bz else 1 - xg
        fit += ce[bz * p, by * p, bx * p] * wz[:, None, None] * wy[None, :, None] * wx[None, None, :]
    assert np.abs(ce - fit).max() <= 1e-10 * np.abs(zs).max()
    s.close()
