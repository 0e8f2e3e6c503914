"""Learned per-patch correction of the LOR V-cycle (oracle; FP64).

The learned form: after the V(1,1) cycle on an interior vertex patch
(Section 3.3, level 0 of the patch), a small convolutional network N maps the
remaining residual t = r - A_j x to a correction of x.  With s = diag(A_j)^(-1/2),
rho = rms(s * t) and the feature f = log(diag(A_j) / mean(diag(A_j))):
    input  (2 channels) = [s * t / rho, f]
    N = conv3^3(2->16) - ReLU - conv3^3(16->16) - ReLU - conv3^3(16->1)
        (3x3x3 kernels, zero padding at the patch boundary, biases)
    x <- x + rho * s * N(input)
so the correction is 1-homogeneous in t.  Training minimises, over pairs
(t, delta) made by the plain V-cycle (delta = e - x, t = A_j delta for a random
error e), the normalised energy of the error left after the correction:
    L = (delta - c)^T A_j (delta - c) / (delta^T A_j delta),  c = rho s N(.).
Weights taps are ordered (dz+1)*9 + (dy+1)*3 + (dx+1); a tap reads the input at
v + (dx, dy, dz) (cross-correlation).  Boxes are (C, B, A) = (z, y, x) arrays.
"""
from __future__ import annotations

import numpy as np

CH = 16
TAPS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def init_params(seed=0, scale=0.1):
    """Seeded weights of the 3-layer network; the last layer starts at zero, so the
    untrained correction is zero and the plain V-cycle result is unchanged."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((CH, 2, 27)) * scale, "b1": np.zeros(CH),
        "W2": rng.standard_normal((CH, CH, 27)) * scale / 4, "b2": np.zeros(CH),
        "W3": np.zeros((1, CH, 27)), "b3": np.zeros(1),
    }


def shift(x, dx, dy, dz):
    """out[..., k, j, i] = x[..., k+dz, j+dy, i+dx] with zeros outside."""
    out = np.zeros_like(x)
    C, B, A = x.shape[-3:]
    src = [slice(max(d, 0), n + min(d, 0)) for d, n in ((dz, C), (dy, B), (dx, A))]
    dst = [slice(max(-d, 0), n + min(-d, 0)) for d, n in ((dz, C), (dy, B), (dx, A))]
    out[(...,) + tuple(dst)] = x[(...,) + tuple(src)]
    return out


def conv(x, W, b):
    """x (Cin, C, B, A), W (Cout, Cin, 27), b (Cout,) -> (Cout, C, B, A)."""
    out = np.zeros((W.shape[0],) + x.shape[1:])
    for t, (dx, dy, dz) in enumerate(TAPS):
        xs = shift(x, dx, dy, dz)
        out += np.einsum("oi,i...->o...", W[:, :, t], xs)
    return out + b[:, None, None, None]


def conv_backward(x, W, g):
    """Gradients of sum(g * conv(x, W, b)) w.r.t. x, W, b."""
    dW = np.zeros_like(W)
    dx = np.zeros_like(x)
    for t, (dxs, dys, dzs) in enumerate(TAPS):
        xs = shift(x, dxs, dys, dzs)
        dW[:, :, t] = np.einsum("ozyx,izyx->oi", g, xs)
        dx += shift(np.einsum("oi,o...->i...", W[:, :, t], g), -dxs, -dys, -dzs)
    return dx, dW, g.sum(axis=(1, 2, 3))


def features(t, diag):
    """Input channels: the D^{-1/2}-scaled residual normalised by its RMS (which makes
    the correction 1-homogeneous in t) and log(diag A_j / its mean); also the scales."""
    s = 1.0 / np.sqrt(diag)
    st = s * t
    rho = np.sqrt(np.mean(st ** 2))
    f = np.log(diag / np.mean(diag))
    return np.stack([st / rho, f]), s, rho


def forward(P, t, diag, act="fp64"):
    """Correction c (same shape as t) and the cache for backward.

    act="bf16": the arithmetic of a bf16 implementation with FP32 (here FP64)
    accumulation, which stores the network's input features and its pre-activations
    in bfloat16: each layer's input is rounded to bf16 (the features; relu of the
    rounded pre-activations is already bf16), the output layer is not."""
    rnd = bf16_round if act == "bf16" else (lambda a: a)
    x0, s, rho = features(t, diag)
    x0 = rnd(x0)
    z1 = rnd(conv(x0, P["W1"], P["b1"]))
    a1 = np.maximum(z1, 0)
    z2 = rnd(conv(a1, P["W2"], P["b2"]))
    a2 = np.maximum(z2, 0)
    y = conv(a2, P["W3"], P["b3"])[0]
    return rho * s * y, (x0, z1, a1, z2, a2, s, rho)


def loss_and_grad(P, t, delta, apply_A, diag, act="fp64"):
    """L for one patch and dL/dparams.  apply_A(v) applies A_j to a box-shaped v.
    act="bf16" also rounds the back-propagated gradients to bf16 where such an
    implementation stores them: the output gradient and the gradients behind each
    ReLU."""
    rnd = bf16_round if act == "bf16" else (lambda a: a)
    c, (x0, z1, a1, z2, a2, s, rho) = forward(P, t, diag, act)
    d = delta - c
    Ad = apply_A(d)
    norm = float(np.sum(delta * t))          # delta^T A delta, since t = A delta
    L = float(np.sum(d * Ad)) / norm
    gy = rnd((-2.0 * rho * s * Ad / norm)[None])
    ga2, gW3, gb3 = conv_backward(a2, P["W3"], gy)
    gz2 = rnd(ga2 * (z2 > 0))
    ga1, gW2, gb2 = conv_backward(a1, P["W2"], gz2)
    gz1 = rnd(ga1 * (z1 > 0))
    _, gW1, gb1 = conv_backward(x0, P["W1"], gz1)
    return L, {"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3}


def bf16_round(a):
    """Round-to-nearest-even to bfloat16, returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
