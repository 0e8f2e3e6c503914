"""C-ABI checks that need no GPU: the library builds, loads, exports every
function declared in include/lor.h, and rejects invalid input on the host."""
import ctypes
import os

import numpy as np
import pytest

from paper_1908_07071_gb300 import lor
from paper_1908_07071_gb300.build import build_library
from paper_1908_07071_gb300.synthetic import make_mesh


@pytest.fixture(scope="module")
def lib():
    build_library()
    return lor.load()


def test_exports_every_declared_symbol(lib):
    names = lor.header_functions()
    assert len(names) >= 12, names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in lor.h but not exported"


def _create(lib, opt, verts, kappa):
    ctx = ctypes.c_void_p()
    st = lib.lor_create(ctypes.byref(ctx), ctypes.byref(opt), verts.ctypes.data_as(ctypes.c_void_p),
                        kappa.ctypes.data_as(ctypes.c_void_p), None)
    return st, ctx


def test_create_validates_on_host(lib):
    verts, kappa = make_mesh(3, 2, seed=0)
    opt = lor.Options()
    lib.lor_default_options(ctypes.byref(opt))
    opt.nx = opt.ny = opt.nz = 2
    st, ctx = _create(lib, opt, verts, kappa)
    assert st == lor.LOR_OK and ctx.value
    lib.lor_destroy(ctx)
    assert opt.weighting == 0                       # the paper's unit patch weights by default
    for field, bad in (("p", 0), ("p", 9), ("dim", 4), ("nx", 0), ("rtol", 0.0), ("max_it", 0),
                       ("weighting", 3), ("weighting", -1)):
        o = lor.Options()
        ctypes.memmove(ctypes.byref(o), ctypes.byref(opt), ctypes.sizeof(o))
        setattr(o, field, bad)
        assert _create(lib, o, verts, kappa)[0] == lor.LOR_EINVAL, field
    bad_kappa = kappa.copy()
    bad_kappa.flat[3] = -1.0
    assert _create(lib, opt, verts, bad_kappa)[0] == lor.LOR_EINVAL
    nan_verts = verts.copy()
    nan_verts.flat[5] = np.nan
    assert _create(lib, opt, nan_verts, kappa)[0] == lor.LOR_EINVAL
    # element counts beyond the kernels' int index range are refused before any array is read
    big = lor.Options()
    ctypes.memmove(ctypes.byref(big), ctypes.byref(opt), ctypes.sizeof(big))
    big.nx = big.ny = big.nz = 1300                      # 2.2e9 elements
    assert _create(lib, big, verts, kappa)[0] == lor.LOR_EINVAL


def test_calls_before_setup_are_rejected(lib):
    verts, kappa = make_mesh(2, 2, seed=0)
    opt = lor.Options()
    lib.lor_default_options(ctypes.byref(opt))
    opt.dim, opt.nx, opt.ny = 2, 2, 2
    st, ctx = _create(lib, opt, verts, kappa)
    assert st == lor.LOR_OK
    assert lib.lor_apply_A(ctx, None, None, 0) == lor.LOR_ESTATE
    assert lib.lor_pcg_solve(ctx, None, None, None, None) == lor.LOR_ESTATE
    assert b"setup" in lib.lor_last_error(ctx)
    assert lib.lor_device_status(ctx) == lor.LOR_ESTATE
    assert lib.lor_selftest_wait(ctx, 16) == lor.LOR_ESTATE
    nb = ctypes.c_size_t(0)
    assert lib.lor_pcg_state_size(ctx, ctypes.byref(nb)) == lor.LOR_ESTATE
    buf = np.zeros(64, dtype=np.uint8)
    vp = ctypes.c_void_p
    assert lib.lor_pcg_state_save(ctx, None, buf.ctypes.data_as(vp), 64) == lor.LOR_ESTATE
    assert lib.lor_pcg_resume(ctx, buf.ctypes.data_as(vp), 64, None, None, None, None) == lor.LOR_ESTATE
    # option switches are host state and may precede setup; bad values are refused
    assert lib.lor_set_weighting(ctx, 1) == lor.LOR_OK
    assert lib.lor_set_weighting(ctx, 3) == lor.LOR_EINVAL
    lib.lor_destroy(ctx)


@pytest.mark.parametrize("dim,n,p", [(2, (3, 2), 3), (3, (2, 1, 2), 2)])
def test_coefficient_points_match_the_oracle_quadrature(lib, dim, n, p):
    """lor_coefficient_points (host only) lists the Gauss points of K_p per element and the
    2-point Gauss points of every LOR sub-cell in the documented order; the oracle computes
    the same points from its own element maps."""
    import itertools
    from oracle import cg
    from oracle.basis import gauss_legendre
    from oracle.mesh import Mesh, multilinear
    verts, kappa = make_mesh(dim, n, seed=6, perturb=0.15)
    opt = lor.Options()
    lib.lor_default_options(ctypes.byref(opt))
    nn = list(n) + [1] * (3 - len(n))
    opt.dim, opt.p, opt.nx, opt.ny, opt.nz = dim, p, nn[0], nn[1], nn[2]
    st, ctx = _create(lib, opt, verts, kappa)
    assert st == lor.LOR_OK
    xq, xh = lor.coefficient_points(lib, ctx, dim)
    m = Mesh(verts, kappa)
    x1, w1 = gauss_legendre(p + 1)
    pts, _ = cg.tensor_points(dim, x1, w1)
    ref_q = np.concatenate([m.element_map(e, pts, p)[0] for e in m.elements()])
    np.testing.assert_allclose(xq, ref_q, atol=1e-14)
    N = cg.node_shape(m.n, p)
    X = cg.node_coordinates(m, p)
    g = 0.5 - 0.5 / np.sqrt(3.0)
    ref_h = []
    for cell in itertools.product(*[range(v - 1) for v in reversed(N)]):
        c = cell[::-1]                                             # (ox, oy[, oz]), x fastest
        corners = []
        for t in range(2 ** dim):
            idx, stride = 0, 1
            for a in range(dim):
                idx += (c[a] + ((t >> a) & 1)) * stride
                stride *= N[a]
            corners.append(X[idx])
        for gi in range(2 ** dim):
            xi = np.array([[g, 1 - g][(gi >> a) & 1] for a in range(dim)])
            ref_h.append(multilinear(np.array(corners), xi[None, :])[0][0])
    np.testing.assert_allclose(xh, np.array(ref_h), atol=1e-14)
    # values: positive and finite only, and CG contexts only
    bq, bh = np.ones(len(xq)), np.ones(len(xh))
    bad = bh.copy()
    bad[3] = 0.0
    vp = ctypes.c_void_p
    assert lib.lor_set_coefficient(ctx, bq.ctypes.data_as(vp), bad.ctypes.data_as(vp)) == lor.LOR_EINVAL
    assert lib.lor_set_coefficient(ctx, None, bh.ctypes.data_as(vp)) == lor.LOR_EINVAL
    assert lib.lor_set_coefficient(ctx, bq.ctypes.data_as(vp), bh.ctypes.data_as(vp)) == lor.LOR_OK
    lib.lor_destroy(ctx)
    if dim == 3:
        opt.disc, opt.eta = lor.LOR_DG_IP, 10.0
        st, ctx = _create(lib, opt, verts, kappa)
        assert st == lor.LOR_OK
        assert lib.lor_set_coefficient(ctx, bq.ctypes.data_as(vp), bh.ctypes.data_as(vp)) == lor.LOR_EINVAL
        lib.lor_destroy(ctx)


def test_node_coordinates_validation(lib):
    """lor_set_node_coordinates (curved elements): finite values, CG only, not together
    with pointwise coefficients; all checked on the host before setup."""
    verts, kappa = make_mesh(2, 2, seed=0)
    opt = lor.Options()
    lib.lor_default_options(ctypes.byref(opt))
    opt.dim, opt.p, opt.nx, opt.ny = 2, 3, 2, 2
    ntot = 7 * 7
    vp = ctypes.c_void_p
    X = np.zeros(2 * ntot)
    st, ctx = _create(lib, opt, verts, kappa)
    bad = X.copy()
    bad[5] = np.inf
    assert lib.lor_set_node_coordinates(ctx, bad.ctypes.data_as(vp)) == lor.LOR_EINVAL
    assert lib.lor_set_node_coordinates(ctx, None) == lor.LOR_EINVAL
    assert lib.lor_set_node_coordinates(ctx, X.ctypes.data_as(vp)) == lor.LOR_OK
    xq, xh = lor.coefficient_points(lib, ctx, 2)
    bq, bh = np.ones(len(xq)), np.ones(len(xh))
    assert lib.lor_set_coefficient(ctx, bq.ctypes.data_as(vp), bh.ctypes.data_as(vp)) == lor.LOR_EINVAL
    lib.lor_destroy(ctx)
    st, ctx = _create(lib, opt, verts, kappa)
    assert lib.lor_set_coefficient(ctx, bq.ctypes.data_as(vp), bh.ctypes.data_as(vp)) == lor.LOR_OK
    assert lib.lor_set_node_coordinates(ctx, X.ctypes.data_as(vp)) == lor.LOR_EINVAL
    lib.lor_destroy(ctx)


C_PROGRAM = r"""
#include <stdio.h>
#include "lor.h"

int main(void) {
  lor_options o;
  lor_default_options(&o);
  o.dim = 2; o.p = 3; o.nx = 2; o.ny = 2;
  double verts[2 * 9], kappa[4] = {1, 1, 1, 1};
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i) { verts[j * 3 + i] = 0.5 * i; verts[9 + j * 3 + i] = 0.5 * j; }
  lor_ctx* ctx = NULL;
  lor_status st = lor_create(&ctx, &o, verts, kappa, NULL);
  long long nq = 0, nh = 0;
  if (st == LOR_OK) st = lor_coefficient_sizes(ctx, &nq, &nh);
  printf("%d %lld %lld\n", (int)st, nq, nh);
  lor_destroy(ctx);
  return st == LOR_OK ? 0 : 1;
}
"""


def test_header_is_c99_and_links_from_c(lib, tmp_path):
    """include/lor.h compiles as strict C99 and the library links and answers from C
    (host-only calls: options, context creation, coefficient sizes)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1908_07071_gb300.build import LIB
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(LIB)
    cmd = [gcc, "-std=c99", "-pedantic", "-Wall", "-Werror", "-I", os.path.join(root, "include"), str(src),
           "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(LIB), "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.split() == ["0", str(4 * 16), str(36 * 4)]


def test_quadrature_points_match_the_oracle_element_maps(lib):
    """lor_quadrature_points (host only, before setup) lists the (p+1)^d Gauss points of every
    element in the order lor_rhs_f reads f: elements x fastest, q = qx + Q qy + Q^2 qz; on
    multilinear elements they are the oracle's multilinear maps of the Gauss points, on curved
    elements the oracle's isoparametric maps (Section 4.2's curved mesh stand-in)."""
    from oracle import cg
    from oracle.basis import gauss_legendre
    from oracle.mesh import Mesh
    from paper_1908_07071_gb300.synthetic import make_quarter_hole_mesh
    cases = []
    v3, k3 = make_mesh(3, (2, 3, 2), seed=2, perturb=0.15)
    cases.append((Mesh(v3, k3), 3, None))
    vq, kq, warp = make_quarter_hole_mesh(4)
    mq = Mesh(vq, kq, warp=warp)
    cases.append((mq, 4, cg.node_coordinates(mq, 4)))
    for m, p, X in cases:
        opt = lor.Options()
        lib.lor_default_options(ctypes.byref(opt))
        opt.dim, opt.p = m.dim, p
        opt.nx, opt.ny = m.n[0], m.n[1]
        opt.nz = m.n[2] if m.dim == 3 else 1
        st, ctx = _create(lib, opt, np.ascontiguousarray(m.vertices), np.ascontiguousarray(m.kappa))
        assert st == lor.LOR_OK
        if X is not None:
            Xs = np.ascontiguousarray(X.T)
            assert lib.lor_set_node_coordinates(ctx, Xs.ctypes.data_as(ctypes.c_void_p)) == lor.LOR_OK
        Q = p + 1
        nq = m.nel * Q ** m.dim
        xq = np.empty(nq * m.dim)
        assert lib.lor_quadrature_points(ctx, xq.ctypes.data_as(ctypes.c_void_p)) == lor.LOR_OK
        xq = xq.reshape(m.nel, Q ** m.dim, m.dim)
        x1, w1 = gauss_legendre(Q)
        pts, _ = cg.tensor_points(m.dim, x1, w1)
        for ie, e in enumerate(m.elements()):
            Xo, _ = m.element_map(e, pts, p)
            np.testing.assert_allclose(xq[ie], Xo, atol=1e-13)
        assert lib.lor_quadrature_points(ctx, None) == lor.LOR_EINVAL
        lib.lor_destroy(ctx)
