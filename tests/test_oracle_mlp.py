"""Pins of the surrogate network's oracle against facts other than itself:
central finite differences of the loss, closed forms of SiLU and of a network
whose hidden weights are zero, the first Adam step, bfloat16 rounding of
exactly representable and tie cases, and hand-computed features."""
import numpy as np
import pytest

from oracle import mlp


def random_params(rng, scale=0.3):
    return rng.normal(0.0, scale, mlp.NPARAM)


def test_layout_size():
    assert mlp.NPARAM == 9349
    p = np.arange(mlp.NPARAM, dtype=np.float64)
    assert np.array_equal(mlp.pack(mlp.unpack(p)), p)
    assert mlp.unpack(p)["W2"][1, 0] == 64 * 10 + 64 + 64  # row-major out x in after W1, b1


def test_silu_and_its_derivative():
    z = np.linspace(-8, 8, 101)
    assert mlp.silu(np.array([0.0]))[0] == 0.0
    assert np.allclose(mlp.silu(np.array([30.0])), 30.0, rtol=1e-12)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.silu_grad(z))) < 1e-8


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    p = random_params(rng)
    X = rng.normal(size=(7, mlp.IN))
    T = rng.normal(size=(7, mlp.OUT))
    L, g = mlp.loss_grad(p, X, T)
    assert L == pytest.approx(np.mean((mlp.forward(p, X) - T) ** 2), rel=1e-14)
    # every bias and output weight, plus a random sample of the other weights
    idx = np.concatenate([np.arange(9024, mlp.NPARAM), np.arange(640, 704), rng.choice(9024, 300, replace=False)])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (mlp.loss_grad(p + e, X, T)[0] - mlp.loss_grad(p - e, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (abs(g[i]) + 1e-3), (i, fd, g[i])


def test_zero_hidden_weights_closed_form():
    rng = np.random.default_rng(1)
    w = mlp.unpack(random_params(rng))
    w["W1"][:] = 0.0
    w["W2"][:] = 0.0
    w["W3"][:] = 0.0
    X = rng.normal(size=(5, mlp.IN))
    Y = mlp.forward(mlp.pack(w), X)
    expect = w["W4"] @ mlp.silu(w["b3"]) + w["b4"]
    assert np.allclose(Y, expect[None, :], rtol=0, atol=1e-14)


def test_first_adam_step_moves_by_lr_times_sign():
    rng = np.random.default_rng(2)
    p = rng.normal(size=mlp.NPARAM)
    g = rng.normal(size=mlp.NPARAM)
    p1, m, v = mlp.adam(p, g, np.zeros_like(p), np.zeros_like(p), 1, 1e-3, eps=0.0)
    assert np.allclose(p1 - p, -1e-3 * np.sign(g), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding_cases():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -2.5, 3.0, 0.0, 65280.0],
                 np.float32)
    r = mlp.bf16_round(x)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa wins (1);
    # 1 + 3 2^-8 is a tie between 1 + 2^-7 and 1 + 2^-6: even wins (1 + 2^-6)
    assert r.tolist() == [1.0, 1.0, 1 + 2 ** -6, 1 + 2 ** -7, -2.5, 3.0, 0.0, 65280.0]


def test_features_by_hand():
    d, k, eps = np.array([0.5, 1e-9]), np.array([0.02, 0.01]), np.array([0.004, 0.002])
    grad = np.array([[1.0, 2.0, 3.0, 4.0], [0.0, -1.0, 0.5, 0.0]])
    R = np.array([[0.01, 0.006, 0.004, -0.002, 0.0, 0.0], [0.005, 0.003, 0.002, 0.001, 0.0, 0.0]])
    F = mlp.features(d, k, eps, grad, R)
    assert F.shape == (2, 10)
    assert F[0, 0] == pytest.approx(np.log(0.5)) and F[1, 0] == pytest.approx(np.log(1e-6))
    assert F[0, 3:7].tolist() == pytest.approx([5.0, 10.0, 15.0, 20.0])  # k/eps = 5
    assert F[0, 7:].tolist() == pytest.approx([0.5, -0.1, 0.3])
    assert mlp.targets(np.ones((2, 5)), eps)[1].tolist() == pytest.approx([500.0] * 5)


def test_bf16_activation_mode_closed_form():
    """With zero hidden weights the bf16-operand network is W4 bf16(SiLU(b3)) + b4
    (bf16-rounded W4), whatever the inputs."""
    rng = np.random.default_rng(8)
    w = mlp.unpack(random_params(rng))
    w["W1"][:] = 0.0
    w["W2"][:] = 0.0
    w["W3"][:] = 0.0
    p = mlp.pack(w).astype(np.float32)
    X = rng.normal(size=(4, mlp.IN))
    Y = mlp.forward(p, X, bf16=True, bf16_act=True)
    wq = mlp.unpack(mlp.bf16_round(p).astype(np.float64))
    a3 = mlp.bf16_round(mlp.silu(wq["b3"]).astype(np.float32)).astype(np.float64)
    assert np.allclose(Y, (wq["W4"] @ a3 + wq["b4"])[None, :], rtol=0, atol=1e-12)
    # and it differs from the FP32-activation network by about a bf16 ulp
    Yf = mlp.forward(p, X, bf16=True)
    assert 0 < np.max(np.abs(Y - Yf)) < 0.05 * np.max(np.abs(Yf))


def test_bf16_gradient_closed_form_with_zero_hidden_weights():
    """With W1 = W2 = W3 = 0 every hidden activation is a constant row:
    a_l = bf16(SiLU(b_l)). The mixed-precision gradients of the top two
    layers then have closed forms in the rounded quantities: with
    dY = bf16(2 (Y - T) / 5n), gW4 = (sum_r dY_r) a3^T, gb4 = sum_r dY_r,
    dz3 = bf16((dY bf16(W4)) * SiLU'(b3)), gW3 = (sum_r dz3_r) a2^T,
    gb3 = sum_r dz3_r."""
    rng = np.random.default_rng(9)
    w = mlp.unpack(random_params(rng))
    w["W1"][:] = 0.0
    w["W2"][:] = 0.0
    w["W3"][:] = 0.0
    p = mlp.pack(w).astype(np.float32).astype(np.float64)
    n = 6
    X = rng.normal(size=(n, mlp.IN))
    T = rng.normal(size=(n, mlp.OUT))
    L, g = mlp.loss_grad(p, X, T, bf16=True)
    q = mlp.unpack(p)
    rb = lambda a: mlp.bf16_round(np.asarray(a, np.float32)).astype(np.float64)
    a2, a3 = rb(mlp.silu(q["b2"])), rb(mlp.silu(q["b3"]))
    W4 = rb(q["W4"])
    Y = np.tile(W4 @ a3 + q["b4"], (n, 1))
    dY = rb(2.0 * (Y - T) / (5 * n))
    dz3 = rb((dY @ W4) * mlp.silu_grad(q["b3"])[None, :])
    G = mlp.unpack(g)
    assert L == pytest.approx(np.sum((Y - T) ** 2) / (5 * n), rel=1e-14)
    assert np.allclose(G["W4"], np.outer(dY.sum(0), a3), rtol=1e-14, atol=1e-300)
    assert np.allclose(G["b4"], dY.sum(0), rtol=1e-14, atol=1e-300)
    assert np.allclose(G["W3"], np.outer(dz3.sum(0), a2), rtol=1e-14, atol=1e-300)
    assert np.allclose(G["b3"], dz3.sum(0), rtol=1e-14, atol=1e-300)


def test_bf16_gradient_is_the_exact_one_within_bf16_rounding():
    """The mixed-precision gradient differs from the exact one, by a few
    bfloat16 ulps of the gradient's scale at most."""
    rng = np.random.default_rng(10)
    p = random_params(rng).astype(np.float32).astype(np.float64)
    X = rng.normal(size=(40, mlp.IN))
    T = rng.normal(size=(40, mlp.OUT))
    L0, g0 = mlp.loss_grad(p, X, T)
    L1, g1 = mlp.loss_grad(p, X, T, bf16=True)
    d = np.max(np.abs(g1 - g0)) / np.max(np.abs(g0))
    assert 0 < d < 8 * 2.0 ** -8
    assert L1 == pytest.approx(L0, rel=0.05)
