"""Pins of the FP64 MLP oracle against facts fixed outside it: bfloat16 rounding against
PyTorch's FP32 -> bfloat16 conversion and hand-worked ties, GELU against values of the
normal CDF and its symmetry, the forward pass against a closed form through one chain of
units, the backward pass against central finite differences of the loss, and Adam against
its closed form under a constant gradient."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M

torch = pytest.importorskip("torch")


def test_bf16_round_matches_torch_and_ties():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-30, 30, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16_round(x.astype(np.float64)), ref)
    # hand-worked ties (8 significant bits): 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    # and goes to the even significand 1; 1 + 3 2^-8 goes to 1 + 2^-6
    assert M.bf16_round(1 + 2.0 ** -8) == 1.0
    assert M.bf16_round(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6
    assert M.bf16_round(-(1 + 3 * 2.0 ** -8)) == -(1 + 2.0 ** -6)
    assert M.bf16_round(1 + 2.0 ** -8 + 2.0 ** -30) == 1 + 2.0 ** -7
    assert M.bf16_round(0.0) == 0.0
    assert M.bf16_round(2.0 ** -130) == 2.0 ** -130        # subnormal, exact
    assert M.bf16_round(3 * 2.0 ** -134) == 2.0 ** -132     # tie below the normal range


def test_gelu_values_symmetry_and_derivative():
    # Phi(1) and Phi(2) of the standard normal distribution
    assert abs(M.gelu(1.0) - 0.8413447460685429) < 1e-15
    assert abs(M.gelu(2.0) - 2 * 0.9772498680518208) < 1e-15
    assert M.gelu(0.0) == 0.0
    z = np.linspace(-6, 6, 241)
    # Phi(z) + Phi(-z) = 1  =>  gelu(z) - gelu(-z) = z
    assert np.max(np.abs(M.gelu(z) - M.gelu(-z) - z)) < 1e-14
    h = 1e-5
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - M.gelu_grad(z))) < 1e-9


def test_forward_single_chain_closed_form():
    """Only one chain of units carries signal: input 0 -> unit 3 -> unit 7 -> unit 1 ->
    unit 250 -> output 65.  A transposed or misplaced weight sends it elsewhere."""
    theta = np.zeros(M.n_params())
    L = M.unpack(theta)
    L[0][0][3, 0] = 1.0
    L[1][0][7, 3] = 1.0
    L[2][0][1, 7] = 1.0
    L[3][0][250, 1] = 1.0
    L[4][0][65, 250] = 2.0
    L[4][1][65] = 0.5
    X = np.zeros((3, 5))
    X[:, 0] = [-1.25, 0.3, 2.0]
    X[:, 1] = 7.0                       # ignored by the chain
    Y, _ = M.forward(theta, X, bf16=False)
    g = M.gelu
    expect = 2.0 * g(g(g(g(X[:, 0])))) + 0.5
    assert np.allclose(Y[:, 65], expect, rtol=0, atol=1e-15)
    Y[:, 65] = 0
    assert np.all(Y == 0)


@pytest.mark.parametrize("dims", [(5, 7, 6, 5, 4, 3), M.DIMS])
def test_backward_matches_finite_differences(dims):
    rng = np.random.default_rng(7)
    n = M.n_params(dims)
    theta = np.concatenate([rng.uniform(-s, s, k) for s, k in
                            ((1.5 / math.sqrt(dims[l]), dims[l + 1] * (dims[l] + 1)) for l in range(len(dims) - 1))])
    X = rng.uniform(-1, 1, (4, dims[0]))
    T = rng.standard_normal((4, dims[-1]))
    L0, grad = M.backward(theta, X, T, bf16=False, dims=dims)
    assert abs(L0 - M.loss(M.forward(theta, X, False, dims)[0], T)) == 0.0
    idx = np.arange(n) if n < 400 else rng.choice(n, 300, replace=False)
    # include every bias of the first and last layers
    idx = np.unique(np.concatenate([idx, np.arange(dims[0] * dims[1], dims[0] * dims[1] + dims[1]),
                                    np.arange(n - dims[-1], n)]))
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (M.loss(M.forward(tp, X, False, dims)[0], T) - M.loss(M.forward(tm, X, False, dims)[0], T)) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(1.0, abs(grad[k])) + 1e-9, k


def test_bf16_gradient_close_to_exact():
    rng = np.random.default_rng(3)
    theta = rng.uniform(-0.1, 0.1, M.n_params())
    X = rng.uniform(-1, 1, (64, 5))
    T = rng.standard_normal((64, 66))
    _, g64 = M.backward(theta, X, T, bf16=False)
    _, g16 = M.backward(theta, X, T, bf16=True)
    assert np.linalg.norm(g16 - g64) / np.linalg.norm(g64) < 2e-2


def test_adam_constant_gradient_closed_form():
    """Under a constant gradient g the bias-corrected moments are exactly g and g^2, so
    every step moves each parameter by -lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th = np.array([1.0, 1.0, 1.0, 1.0])
    m, v = np.zeros(4), np.zeros(4)
    lr, eps = 1e-2, 1e-8
    for s in range(1, 6):
        before = th.copy()
        M.adam(th, g, m, v, s, lr, eps=eps)
        assert np.allclose(th - before, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-18)
