"""Pins of the surrogate-network oracle: finite differences, and independent
library routines (torch CPU, fp64) for the forward pass, GELU, BF16 rounding
and Adam.  CPU only."""
import numpy as np
import pytest
import torch

from oracle import mlp

SMALL = (7, 5, 4, 3)


def rand_theta(dims, seed=0, scale=0.5):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, mlp.n_params(dims))


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    a = (rng.normal(0, 1, 10000) * 10.0 ** rng.integers(-20, 20, 10000)).astype(np.float32)
    # include exact ties
    a[:4] = np.array([1.00390625, 1.01171875, -3.0078125, 65535.0], np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(a), ref)


def test_forward_matches_torch_fp64():
    dims = SMALL
    th = rand_theta(dims, 1)
    X = np.random.default_rng(2).normal(0, 1, (9, dims[0]))
    y = mlp.forward(th, X, dims, bf16=False)
    h = torch.from_numpy(X)
    for i, (W, b) in enumerate(mlp.unpack(th, dims)):
        h = torch.nn.functional.linear(h, torch.from_numpy(W.copy()), torch.from_numpy(b.copy()))
        if i < len(dims) - 2:
            h = torch.nn.functional.gelu(h, approximate="none")
    assert np.allclose(y, h.numpy(), rtol=1e-13, atol=1e-14)


def test_gradient_by_finite_differences():
    dims = SMALL
    th = rand_theta(dims, 3)
    rng = np.random.default_rng(4)
    X, T = rng.normal(0, 1, (6, dims[0])), rng.normal(0, 1, (6, dims[-1]))
    L, g = mlp.loss_and_grad(th, X, T, dims, bf16=False)
    eps = 1e-6
    for k in rng.choice(len(th), 25, replace=False):
        tp, tm = th.copy(), th.copy()
        tp[k] += eps; tm[k] -= eps
        fd = (mlp.loss_and_grad(tp, X, T, dims, False)[0] - mlp.loss_and_grad(tm, X, T, dims, False)[0]) / (2 * eps)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_gradient_matches_torch_autograd():
    dims = SMALL
    th = rand_theta(dims, 5)
    rng = np.random.default_rng(6)
    X, T = rng.normal(0, 1, (8, dims[0])), rng.normal(0, 1, (8, dims[-1]))
    L, g = mlp.loss_and_grad(th, X, T, dims, bf16=False)
    params = [torch.tensor(p.copy(), requires_grad=True) for Wb in mlp.unpack(th, dims) for p in Wb]
    h = torch.from_numpy(X)
    for i in range(len(dims) - 1):
        h = torch.nn.functional.linear(h, params[2 * i], params[2 * i + 1])
        if i < len(dims) - 2:
            h = torch.nn.functional.gelu(h)
    loss = torch.nn.functional.mse_loss(h, torch.from_numpy(T))
    loss.backward()
    gt = np.concatenate([p.grad.numpy().ravel() for p in params])
    assert L == pytest.approx(loss.item(), rel=1e-13)
    assert np.allclose(g, gt, rtol=1e-11, atol=1e-14)


def test_adam_matches_torch():
    th = rand_theta(SMALL, 7)
    rng = np.random.default_rng(8)
    opt = mlp.Adam(th, lr=1e-2)
    p = torch.tensor(th.copy(), requires_grad=True)
    topt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for _ in range(5):
        g = rng.normal(0, 1, th.shape)
        opt.step(g)
        p.grad = torch.from_numpy(g.copy())
        topt.step()
    assert np.allclose(opt.theta, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_bf16_forward_rounds_only_where_stored():
    """BF16 forward equals the FP64 forward applied to rounded input and weights
    when there is a single layer (no hidden activation to round)."""
    dims = (11, 4)
    th = rand_theta(dims, 9)
    X = np.random.default_rng(10).normal(0, 1, (5, 11))
    W, b = mlp.unpack(th, dims)[0]
    expect = mlp.bf16_round(X) @ mlp.bf16_round(W).T + b
    assert np.allclose(mlp.forward(th, X, dims, bf16=True), expect, rtol=1e-14, atol=0)


def test_surrogate_runs_round_trip(tmp_path):
    """Runs written by the study's save_runs come back field for field."""
    from paper_2506_05362_gb300 import surrogate as SG
    rng = np.random.default_rng(0)
    runs = [SG.Run(path=p, n_grains=8 + q, seed=q, strain=rng.normal(size=(5, 6)), stress=rng.normal(size=(5, 6)),
                   desc=rng.normal(size=(5, 13)), pd_seconds=0.5 * q, steps=100 + q, nodes=1000 + q,
                   precompress_steps=7, p_confine=2e6, sf_confine=0.6) for q, p in enumerate(["uniaxial_x", "shear_xy"])]
    f = str(tmp_path / "runs.npz")
    SG.save_runs(f, runs)
    back = SG.load_runs(f)
    assert len(back) == 2
    for a, b in zip(runs, back):
        for k in ("path", "n_grains", "seed", "pd_seconds", "steps", "nodes", "precompress_steps", "p_confine",
                  "sf_confine"):
            assert getattr(a, k) == getattr(b, k)
        for k in ("strain", "stress", "desc"):
            assert np.array_equal(getattr(a, k), getattr(b, k))
