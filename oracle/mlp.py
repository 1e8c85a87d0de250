"""FP64 oracle of the bulk-stress surrogate network -- TEST INFRASTRUCTURE.

The paper motivates a representative-volume surrogate (Sec. 1, Sec. 6.4: the
force per unit area converges with grain count, pointing to RVE use in a
multiscale model) but prints no network.  The network here is the one the
build specifies: an MLP 109 -> 256 -> 256 -> 256 -> 256 -> 6 with GELU between
layers, trained with an MSE loss and Adam.  Readings:
  * GELU is the exact form 0.5 x (1 + erf(x / sqrt 2)) (no tanh approximation).
  * loss = mean over batch and outputs of (y - t)^2.
  * Adam with beta1 = 0.9, beta2 = 0.999, eps = 1e-8 and bias correction.
  * The BF16 variant rounds to nearest-even exactly where the CUDA path stores
    BF16: the network input, the weights, each hidden activation after GELU,
    and, for the backward pass, each hidden pre-activation that GELU' reads.
    Biases, the output and all accumulation stay in high precision.

Parameter layout (flat float32 vector, shared with the library's get/set):
for each layer l in order, W_l row-major (out x in), then b_l (out).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

DIMS = (109, 256, 256, 256, 256, 6)


def bf16_round(a):
    """Round float32 values to bfloat16 (round to nearest, ties to even),
    returned as float64.  NaN/inf are not expected here."""
    f = np.ascontiguousarray(a, np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bias = np.uint64(0x7FFF) + ((bits >> np.uint64(16)) & np.uint64(1))
    r = ((bits + bias) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def n_params(dims=DIMS):
    return sum(dims[i + 1] * dims[i] + dims[i + 1] for i in range(len(dims) - 1))


def unpack(theta, dims=DIMS):
    """Flat vector -> list of (W, b) in float64."""
    theta = np.asarray(theta, np.float64)
    out, k = [], 0
    for i in range(len(dims) - 1):
        fi, fo = dims[i], dims[i + 1]
        W = theta[k:k + fo * fi].reshape(fo, fi); k += fo * fi
        b = theta[k:k + fo]; k += fo
        out.append((W, b))
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def forward(theta, X, dims=DIMS, bf16=True, keep=False):
    """y = MLP(X).  With bf16=True, X, W and hidden activations are rounded to
    BF16 as the CUDA path stores them; arithmetic is FP64."""
    layers = unpack(theta, dims)
    q = bf16_round if bf16 else (lambda a: np.asarray(a, np.float64))
    h = q(X)
    cache = []
    for i, (W, b) in enumerate(layers):
        Wq = q(W)
        z = h @ Wq.T + b
        cache.append((h, Wq, z))
        if i < len(layers) - 1:
            h = q(gelu(z))
        else:
            h = z
    return (h, cache) if keep else h


def loss_and_grad(theta, X, T, dims=DIMS, bf16=True):
    """MSE loss and its gradient with respect to the (unrounded) parameters;
    rounding is treated as the identity in the backward pass."""
    Y, cache = forward(theta, X, dims, bf16, keep=True)
    q = bf16_round if bf16 else (lambda a: a)
    B = X.shape[0]
    diff = Y - T
    loss = float((diff * diff).sum() / (B * dims[-1]))
    g = 2.0 * diff / (B * dims[-1])
    grads = []
    for i in range(len(cache) - 1, -1, -1):
        h, Wq, z = cache[i]
        if i < len(cache) - 1:
            g = g * gelu_grad(q(z))
        gW = g.T @ h
        gb = g.sum(0)
        grads.append((gW, gb))
        g = g @ Wq
    grads.reverse()
    return loss, pack(grads)


class Adam:
    """Adam (Kingma and Ba) on a flat FP64 parameter vector."""

    def __init__(self, theta, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.theta = np.asarray(theta, np.float64).copy()
        self.m = np.zeros_like(self.theta)
        self.v = np.zeros_like(self.theta)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, grad):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * grad
        self.v = self.b2 * self.v + (1 - self.b2) * grad * grad
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        self.theta = self.theta - self.lr * mh / (np.sqrt(vh) + self.eps)
        return self.theta
