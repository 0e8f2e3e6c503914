"""Pins of the learned-correction oracle (no GPU): convolution against a library
correlation, gradients against central finite differences, homogeneity, and the
zero-initialised last layer leaving the V-cycle unchanged."""
import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import learned as L


def test_conv_matches_library_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 4, 5, 6))
    W = rng.standard_normal((3, 2, 27))
    b = rng.standard_normal(3)
    out = L.conv(x, W, b)
    for o in range(3):
        ref = np.full(x.shape[1:], b[o])
        for i in range(2):
            k = W[o, i].reshape(3, 3, 3)            # (dz, dy, dx)
            ref += ndi.correlate(x[i], k, mode="constant", cval=0.0)
        np.testing.assert_allclose(out[o], ref, atol=1e-12)


def _problem(seed=1, shape=(5, 5, 5)):
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    M = rng.standard_normal((n, n)) * 0.1
    A = M @ M.T + np.diag(rng.uniform(1, 2, n))
    diag = np.diag(A).reshape(shape)
    delta = rng.standard_normal(shape)
    t = (A @ delta.ravel()).reshape(shape)
    apply_A = lambda v: (A @ v.ravel()).reshape(shape)  # noqa: E731
    return t, delta, apply_A, diag


def test_gradients_match_finite_differences():
    P = L.init_params(seed=3, scale=0.3)
    P["W3"] = np.random.default_rng(4).standard_normal(P["W3"].shape) * 0.1
    P["b3"] = np.array([0.05])
    t, delta, apply_A, diag = _problem()
    _, G = L.loss_and_grad(P, t, delta, apply_A, diag)
    rng = np.random.default_rng(5)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in P[name].shape)
            h = 1e-6
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name][idx] += h
            Pm[name][idx] -= h
            fd = (L.loss_and_grad(Pp, t, delta, apply_A, diag)[0] - L.loss_and_grad(Pm, t, delta, apply_A, diag)[0]) / (2 * h)
            assert abs(fd - G[name][idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, G[name][idx])


def test_homogeneous_and_zero_init():
    P = L.init_params(seed=0)
    t, delta, apply_A, diag = _problem()
    c, _ = L.forward(P, t, diag)
    assert np.all(c == 0)                       # W3 = 0: plain V-cycle, loss = 1
    Lz, _ = L.loss_and_grad(P, t, delta, apply_A, diag)
    assert abs(Lz - 1.0) < 1e-12
    P["W3"] = np.random.default_rng(1).standard_normal(P["W3"].shape)
    c1, _ = L.forward(P, t, diag)
    c2, _ = L.forward(P, 3.7 * t, diag)
    np.testing.assert_allclose(c2, 3.7 * c1, rtol=1e-12)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.14159])
    r = L.bf16_round(vals)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7 and r[3] == -2.5
    assert abs(r[4] - 3.140625) < 1e-12


def test_bf16_activation_mode():
    """act="bf16" (the arithmetic of the tensor-core kernels): the cached features and
    pre-activations are bfloat16 numbers, and the correction, the loss and the gradient
    stay within the bf16 rounding error of the FP64 mode."""
    P = L.init_params(seed=3, scale=0.3)
    P["W3"] = np.random.default_rng(4).standard_normal(P["W3"].shape) * 0.1
    t, delta, apply_A, diag = _problem(seed=2)
    c64, _ = L.forward(P, t, diag)
    c16, (x0, z1, a1, z2, a2, s, rho) = L.forward(P, t, diag, act="bf16")
    for a in (x0, z1, z2):
        np.testing.assert_array_equal(L.bf16_round(a), a)
    assert np.abs(c16 - c64).max() <= 0.03 * np.abs(c64).max()
    assert np.abs(c16 - c64).max() > 0                       # the rounding is really applied
    L64, G64 = L.loss_and_grad(P, t, delta, apply_A, diag)
    L16, G16 = L.loss_and_grad(P, t, delta, apply_A, diag, act="bf16")
    assert abs(L16 - L64) <= 0.01 * abs(L64)
    # gradients are sums over the patch with cancellation, so compare them as vectors
    g64 = np.concatenate([G64[k].ravel() for k in sorted(G64)])
    g16 = np.concatenate([G16[k].ravel() for k in sorted(G16)])
    assert np.linalg.norm(g16 - g64) <= 0.1 * np.linalg.norm(g64)
    assert g16 @ g64 >= 0.99 * np.linalg.norm(g16) * np.linalg.norm(g64)


@pytest.mark.parametrize("n,p", [(4, 3), (3, 4)])
def test_exact_patch_solves_bound_the_learned_gain(n, p):
    """The learned correction adds to each patch's V-cycle result an estimate of the
    error that cycle leaves on the patch; at best it makes every patch solve exact.
    With exact patch solves the additive preconditioner needs as many PCG iterations
    as with the V(1,1) cycle (within one), so the learned form can shorten the solve
    only through a cheaper cycle, never through fewer iterations."""
    from oracle import cg, krylov
    from oracle import lor as olor
    from oracle.mesh import Mesh
    from paper_1908_07071_gb300.synthetic import make_mesh
    v, k = make_mesh(3, n, seed=11, perturb=0.15)
    m = Mesh(v, k)
    K = cg.assemble_stiffness(m, p)
    N = cg.node_shape(m.n, p)
    b = cg.load_vector(m, p, lambda X: np.ones(len(X)))
    its = []
    for exact in (False, True):
        B = olor.LORPreconditioner(m, p, exact_local=exact)
        its.append(krylov.pcg(lambda u: cg.apply_A(K, N, u), B.apply, b, rtol=1e-8)[1])
    assert abs(its[0] - its[1]) <= 1, its
