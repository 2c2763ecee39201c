"""FP64 CPU oracle of the crater-surrogate MLP.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU leg use this
module; the library never does.

Network (the crater surrogate of this library): 5 normalised impact parameters -> four
hidden layers of 256 units with the GELU activation in its erf form (Hendrycks & Gimpel
2016: gelu(z) = z * Phi(z), Phi the standard normal CDF) -> 66 linear outputs.  Loss: the
mean squared error over all outputs of all samples.  Optimiser: Adam (Kingma & Ba 2015,
Algorithm 1, with the bias-corrected moments).

Parameters are one flat vector, layer by layer: W_l (n_out x n_in, row-major), then b_l.

Rounding.  With ``bf16=True`` the oracle rounds to bfloat16 (round to nearest, ties to
even) exactly the tensors that the GPU kernels hold in bfloat16 -- the inputs, the weights,
the hidden activations gelu(Z) and the back-propagated pre-activation gradients dL/dZ --
and computes every product and sum in FP64.  With ``bf16=False`` nothing is rounded and the
gradients are the exact derivatives of the loss, the form that the finite-difference pins
check.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

DIMS = (5, 256, 256, 256, 256, 66)


def n_params(dims=DIMS) -> int:
    return sum(dims[l + 1] * dims[l] + dims[l + 1] for l in range(len(dims) - 1))


def unpack(theta: np.ndarray, dims=DIMS):
    """Flat vector -> [(W_1, b_1), ..., (W_L, b_L)] as views."""
    out, o = [], 0
    for l in range(len(dims) - 1):
        ni, no = dims[l], dims[l + 1]
        W = theta[o:o + no * ni].reshape(no, ni)
        o += no * ni
        b = theta[o:o + no]
        o += no
        out.append((W, b))
    assert o == theta.size
    return out


def bf16_round(x) -> np.ndarray:
    """Round FP64 values to the nearest bfloat16 (8 significant bits, FP32's exponent
    range), ties to even, returned as FP64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
    # quantum 2^(e - 8) for normal numbers, 2^-133 below bfloat16's normal range
    q = np.maximum(e - 8, -133)
    r = np.ldexp(np.rint(np.ldexp(x, -q)), q)   # np.rint rounds half to even
    return np.where(np.isfinite(x), r, x)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """d gelu / dz = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta: np.ndarray, X: np.ndarray, bf16: bool = True, dims=DIMS):
    """Returns (Y, cache) with cache = (H_0, [Z_1..Z_L], [H_1..H_{L-1}])."""
    rd = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    layers = unpack(np.asarray(theta, dtype=np.float64), dims)
    H = rd(X)
    Hs, Zs = [H], []
    for l, (W, b) in enumerate(layers):
        Z = H @ rd(W).T + b
        Zs.append(Z)
        if l + 1 < len(layers):
            H = rd(gelu(Z))
            Hs.append(H)
    return Zs[-1], (Hs, Zs)


def loss(Y: np.ndarray, T: np.ndarray) -> float:
    return float(np.mean((Y - T) ** 2))


def backward(theta: np.ndarray, X: np.ndarray, T: np.ndarray, bf16: bool = True, dims=DIMS):
    """Loss and its gradient (flat, same layout as theta).  The output gradient
    dL/dY = 2 (Y - T) / (B * n_out); each layer's dL/dZ is rounded (bf16 form) once and that
    rounded tensor gives dW_l = G_l^T H_{l-1}, db_l = sum over samples of G_l and the
    gradient passed down, (G_l W_l) * gelu'(Z_{l-1})."""
    rd = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    theta = np.asarray(theta, dtype=np.float64)
    layers = unpack(theta, dims)
    Y, (Hs, Zs) = forward(theta, X, bf16, dims)
    B = X.shape[0]
    L = loss(Y, T)
    grad = np.zeros_like(theta)
    glayers = unpack(grad, dims)
    dZ = 2.0 * (Y - T) / (B * Y.shape[1])
    for l in range(len(layers) - 1, -1, -1):
        G = rd(dZ)
        gW, gb = glayers[l]
        gW[...] = G.T @ Hs[l]
        gb[...] = G.sum(axis=0)
        if l > 0:
            dZ = (G @ rd(layers[l][0])) * gelu_grad(Zs[l - 1])
    return L, grad


def adam(theta, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place (step counts from 1)."""
    m *= beta1
    m += (1.0 - beta1) * grad
    v *= beta2
    v += (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    theta -= lr * mh / (np.sqrt(vh) + eps)

