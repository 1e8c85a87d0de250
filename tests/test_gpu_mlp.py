"""Surrogate MLP on the GPU (BF16 tensor-core kernels) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

DIMS = (109, 256, 256, 256, 256, 6)
# Tolerances derived from BF16 storage (unit roundoff 2^-9): each of the 5
# layers adds at most about one rounding of the activations it consumes, and a
# rounding decision can flip where FP32 and FP64 accumulation differ by one
# FP32 ulp; the output then differs by O(5 * 2^-9 / sqrt(fan-in)) relative.
FWD_TOL = 4e-3
GRAD_TOL = 3e-2   # gradients also round dZ to BF16 at each layer
# Element-wise bounds, |got - want| <= ATOL * scale + RTOL * |want|, so that one
# wrong row, column or weight cannot hide inside a norm.  A hidden activation
# whose FP32 and FP64 values straddle a BF16 rounding boundary rounds one way on
# the GPU and the other in the oracle: it moves by one BF16 ulp (2^-8 |h|), which
# the next layer spreads over its outputs with weights |W| <= 1.7/16.  FP32
# accumulation over K = 256 terms differs from FP64 by ~sqrt(K) 2^-24 relative,
# so a flip happens with probability ~sqrt(K) 2^-16 per activation: a few flips
# per row of 1024 hidden activations, each moving an output by ~1e-3 of its
# column's RMS; the GELU's erf approximation (absolute error <= 1.5e-7) adds as
# many.  A CPU emulation (FP32 accumulation, BF16 storage) gives at most 1.0e-2
# of the column RMS; the bound takes 5x that.  Gradients round dZ and the
# pre-activations that GELU' reads to BF16 as well (the oracle rounds the latter
# where the kernels store them): the emulation gives at most 2.8e-2 of the
# layer's RMS gradient.
FWD_ATOL, FWD_RTOL = 5e-2, 1e-2      # scale: RMS of the output column
GRAD_ATOL, GRAD_RTOL = 1e-1, 2e-2    # scale: RMS of the layer's W (or b) gradient


@pytest.fixture(scope="module")
def pd():
    import torch
    assert torch.cuda.is_available()
    from paper_2506_05362_gb300 import pd as _pd
    return _pd


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def assert_elementwise_forward(Y, ref):
    """|Y - ref| <= FWD_ATOL * rms(column of ref) + FWD_RTOL * |ref| on every entry."""
    Y = np.asarray(Y, np.float64)
    col = np.sqrt((ref ** 2).mean(0, keepdims=True))
    bad = np.abs(Y - ref) > FWD_ATOL * col + FWD_RTOL * np.abs(ref)
    assert not bad.any(), f"{int(bad.sum())} entries off, first at {np.argwhere(bad)[0]}"


def assert_layers(g, rg):
    """Per layer, the weight gradient and the bias gradient separately: rel-L2 and
    element-wise (scale: the RMS of that block of the oracle's gradient)."""
    off = 0
    for i in range(len(DIMS) - 1):
        nW = DIMS[i + 1] * DIMS[i]
        for what, sl in (("W", slice(off, off + nW)), ("b", slice(off + nW, off + nW + DIMS[i + 1]))):
            a, r = np.asarray(g[sl], np.float64), rg[sl]
            assert rel_l2(a, r) < GRAD_TOL, f"layer {i} {what}"
            rms = np.sqrt((r ** 2).mean())
            bad = np.abs(a - r) > GRAD_ATOL * rms + GRAD_RTOL * np.abs(r)
            assert not bad.any(), f"layer {i} {what}: {int(bad.sum())} entries off"
        off += nW + DIMS[i + 1]


def inputs(batch, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 1, (batch, DIMS[0])).astype(np.float32)
    T = rng.normal(0, 1, (batch, DIMS[-1])).astype(np.float32)
    return X, T


def theta(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(len(DIMS) - 1):
        b = scale / np.sqrt(DIMS[i])
        parts.append(rng.uniform(-b, b, DIMS[i + 1] * DIMS[i]))
        parts.append(rng.uniform(-0.1, 0.1, DIMS[i + 1]))
    return np.concatenate(parts).astype(np.float32)


@pytest.mark.parametrize("path", [2, 1])
@pytest.mark.parametrize("batch", [1, 37, 128, 1003, 4096])
def test_forward_matches_oracle(pd, batch, path):
    """path 2: fused tcgen05 kernel (required); path 1: mma.sync GEMMs."""
    net = pd.MLP(DIMS)
    net.set_forward_path(path)
    th = theta(1, scale=1.7)
    net.set_params(th)
    X, _ = inputs(batch, 2)
    Y = net.forward(X)
    ref = omlp.forward(th.astype(np.float64), X, DIMS, bf16=True)
    assert rel_l2(Y, ref) < FWD_TOL
    assert_elementwise_forward(Y, ref)
    net.close()


@pytest.mark.parametrize("path", [2, 1])
def test_forward_full_batch_sampled(pd, path):
    """Inference batch 65536 in the benchmark's configuration; rows sampled for the oracle."""
    net = pd.MLP(DIMS)
    net.set_forward_path(path)
    th = theta(3, scale=1.7)
    net.set_params(th)
    X, _ = inputs(65536, 4)
    Y = net.forward(X)
    idx = np.random.default_rng(5).choice(65536, 2000, replace=False)
    ref = omlp.forward(th.astype(np.float64), X[idx], DIMS, bf16=True)
    assert rel_l2(Y[idx], ref) < FWD_TOL
    assert_elementwise_forward(Y[idx], ref)
    assert np.all(np.isfinite(Y))


@pytest.mark.parametrize("path", [2, 1])
@pytest.mark.parametrize("batch", [64, 999, 4096])
def test_gradient_matches_oracle(pd, batch, path):
    """path 2: tcgen05 forward and backward GEMMs (required); path 1: mma.sync."""
    net = pd.MLP(DIMS)
    net.set_forward_path(path)
    th = theta(6, scale=1.7)
    net.set_params(th)
    X, T = inputs(batch, 7)
    loss, g = net.grad(X, T)
    rl, rg = omlp.loss_and_grad(th.astype(np.float64), X, T, DIMS, bf16=True)
    assert loss == pytest.approx(rl, rel=FWD_TOL)
    assert rel_l2(g, rg) < GRAD_TOL
    # per layer and per block (W, b), so a wrong layer or bias cannot hide
    assert_layers(g, rg)


def test_adam_update_matches_oracle(pd):
    net = pd.MLP(DIMS)
    th = theta(8)
    net.set_params(th)
    X, T = inputs(512, 9)
    _, g = net.grad(X, T)
    net.train_step(X, T, lr=1e-3)
    opt = omlp.Adam(th.astype(np.float64), lr=1e-3)
    opt.step(g.astype(np.float64))
    assert np.allclose(net.get_params(), opt.theta, rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("path", [2, 1])
def test_training_reduces_loss(pd, path):
    """Fit a smooth map: the loss falls by an order of magnitude."""
    net = pd.MLP(DIMS, seed=3)
    net.set_forward_path(path)
    rng = np.random.default_rng(10)
    X = rng.normal(0, 1, (8192, DIMS[0])).astype(np.float32)
    A = rng.normal(0, 0.2, (DIMS[0], DIMS[-1]))
    T = np.tanh(X @ A).astype(np.float32)
    first = net.train_step(X, T, 1e-3)
    for _ in range(150):
        last = net.train_step(X, T, 1e-3)
    assert last < 0.1 * first


def test_gradient_full_batch_sampled_tc(pd):
    """The benchmark's batch (65,536) on the tcgen05 training path: gradient
    against the oracle evaluated on the same batch (the oracle's FP64 forward
    and backward over 65,536 rows take a few seconds)."""
    net = pd.MLP(DIMS)
    net.set_forward_path(2)
    th = theta(11, scale=1.7)
    net.set_params(th)
    X, T = inputs(65536, 12)
    loss, g = net.grad(X, T)
    rl, rg = omlp.loss_and_grad(th.astype(np.float64), X, T, DIMS, bf16=True)
    assert loss == pytest.approx(rl, rel=FWD_TOL)
    assert rel_l2(g, rg) < GRAD_TOL
    assert_layers(g, rg)
