"""TEST INFRASTRUCTURE ONLY: plain FP64 numpy reference of the learned
surrogate of the elliptic-relaxation solve.

The paper solves Eq. elliptic-relaxation for wp_ij by finite elements every
step (Section 2.2). The optional surrogate maps local node quantities to
wp_ij / eps with a 10 -> 64 -> 64 -> 64 -> 5 network with SiLU activations.
This module writes out that network's forward pass, the mean-squared-error
loss and its gradient by the chain rule, one Adam step (Kingma & Ba 2015),
bfloat16 round-to-nearest-even, and the node features and targets. The
definitions are written from the mathematics, with no blocking or fusion.
Only the test-suite may import it; it shares nothing with the CUDA library.

Parameter layout (flat, row-major, out x in):
  W1[64][10] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[5][64] b4[5]
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 10, 64, 5
SHAPES = (("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
          ("W4", (OUT, H)), ("b4", (OUT,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p) -> dict:
    p = np.asarray(p, np.float64)
    assert p.size == NPARAM
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SHAPES])


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s + z * s * (1.0 - s)


def bf16_round(a) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float32: keep the top 16 bits of the IEEE single after adding half an
    ulp of bfloat16 plus the tie-breaking bit."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    bias = 0x7FFF + ((u >> 16) & 1)
    r = ((u + bias) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def forward(p, X, bf16: bool = False, bf16_act: bool = False):
    """Network output Y[n][5] for standardised inputs X[n][10] (FP64
    arithmetic). bf16=True first rounds the parameters to bfloat16;
    bf16_act=True also rounds the inputs and every hidden activation to
    bfloat16 (the operands of a bf16 tensor-core product), the biases and
    the accumulation staying exact."""
    if bf16:
        p = bf16_round(np.asarray(p, np.float32)).astype(np.float64)
    w = unpack(p)
    r = (lambda a: bf16_round(np.asarray(a, np.float32)).astype(np.float64)) if bf16_act else (lambda a: a)
    X = r(np.asarray(X, np.float64))
    a1 = r(silu(X @ w["W1"].T + w["b1"]))
    a2 = r(silu(a1 @ w["W2"].T + w["b2"]))
    a3 = r(silu(a2 @ w["W3"].T + w["b3"]))
    return a3 @ w["W4"].T + w["b4"]


def loss_grad(p, X, T, bf16: bool = False):
    """L = sum((Y - T)^2) / (5 n) and dL/dp (chain rule, layer by layer).

    bf16=True: the mixed precision of a bfloat16 tensor-core product chain.
    Every operand of a matrix product is rounded to bfloat16 where it enters
    the product (FP32 value first, then bfloat16): the weights, the inputs,
    the hidden activations, dY and each layer's dZ. Bias adds, SiLU and its
    derivative, the loss and every sum stay exact. A bias gradient is the sum
    of the rounded dZ, as the weight-gradient product gives it."""
    w = unpack(p)
    r = (lambda a: bf16_round(np.asarray(a, np.float32)).astype(np.float64)) if bf16 else (lambda a: a)
    W = {k: r(w[k]) for k in ("W1", "W2", "W3", "W4")}
    X = r(np.asarray(X, np.float64))
    T = np.asarray(T, np.float64)
    n = X.shape[0]
    z1 = X @ W["W1"].T + w["b1"]
    a1 = r(silu(z1))
    z2 = a1 @ W["W2"].T + w["b2"]
    a2 = r(silu(z2))
    z3 = a2 @ W["W3"].T + w["b3"]
    a3 = r(silu(z3))
    Y = a3 @ W["W4"].T + w["b4"]
    E = Y - T
    L = float(np.sum(E * E) / (OUT * n))
    dY = r(2.0 * E / (OUT * n))
    g = {"W4": dY.T @ a3, "b4": dY.sum(0)}
    dz3 = r((dY @ W["W4"]) * silu_grad(z3))
    g["W3"], g["b3"] = dz3.T @ a2, dz3.sum(0)
    dz2 = r((dz3 @ W["W3"]) * silu_grad(z2))
    g["W2"], g["b2"] = dz2.T @ a1, dz2.sum(0)
    dz1 = r((dz2 @ W["W2"]) * silu_grad(z1))
    g["W1"], g["b1"] = dz1.T @ X, dz1.sum(0)
    return L, pack(g)


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step with bias correction; returns new (p, m, v)."""
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return np.asarray(p, np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v


def features(d, k, eps, grad, R):
    """Node features: log d (d floored at 1e-6), log k, log eps,
    (k/eps) [dU/dx, dU/dy, dV/dx, dV/dy], [<uu>, <uv>, <vv>] / k.
    R holds uu, vv, ww, uv, uw, vw per node."""
    d = np.maximum(np.asarray(d, np.float64), 1e-6)
    k = np.asarray(k, np.float64)
    eps = np.asarray(eps, np.float64)
    tau = (k / eps)[:, None]
    R = np.asarray(R, np.float64)
    return np.column_stack([np.log(d), np.log(k), np.log(eps), tau * np.asarray(grad, np.float64),
                            R[:, 0] / k, R[:, 3] / k, R[:, 1] / k])


def targets(wp, eps):
    """wp_ij / eps for (11, 12, 21, 22, 33)."""
    return np.asarray(wp, np.float64) / np.asarray(eps, np.float64)[:, None]
