"""Pins for the oracle of the learned drift proposal (oracle/convnet.py).

* strided circular convolution and its backward against torch's CPU conv1d
  (circular padding) and autograd, in FP64;
* the whole network's parameter gradients against central differences;
* the Adam update against torch.optim.Adam on the same gradients.
"""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fn

from oracle import convnet as CN


def test_conv_forward_backward_match_torch():
    r = np.random.default_rng(0)
    x = r.normal(size=(3, 4, 32))
    w = r.normal(size=(6, 4, 5))
    b = r.normal(size=6)
    out = CN.conv_forward(x, w, b)
    xt = torch.tensor(x, requires_grad=True)
    wt = torch.tensor(w, requires_grad=True)
    bt = torch.tensor(b, requires_grad=True)
    ref = Fn.conv1d(Fn.pad(xt, (2, 2), mode="circular"), wt, bt, stride=2)
    assert np.allclose(out, ref.detach().numpy(), atol=1e-12)
    g = r.normal(size=out.shape)
    ref.backward(torch.tensor(g))
    dx, dw, db = CN.conv_backward(x, w, g)
    assert np.allclose(dx, xt.grad.numpy(), atol=1e-12)
    assert np.allclose(dw, wt.grad.numpy(), atol=1e-12)
    assert np.allclose(db, bt.grad.numpy(), atol=1e-12)


def test_network_gradient_matches_central_differences():
    K, Ns, C, n = 4, 3, 8, 64
    p = CN.init_params(C, K, Ns, n, seed=1)
    for k in p:
        if k.startswith("b"):
            p[k] = 0.05 * np.random.default_rng(2).normal(size=p[k].shape)
    r = np.random.default_rng(3)
    x0 = r.normal(size=(2, 2, n))
    target = r.normal(size=(2, Ns, K))
    L, g = CN.loss_and_grad(p, x0, target, K, Ns)
    eps = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in r.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            Lp, _ = CN.loss_and_grad(p, x0, target, K, Ns)
            flat[idx] = old - eps
            Lm, _ = CN.loss_and_grad(p, x0, target, K, Ns)
            flat[idx] = old
            fd = (Lp - Lm) / (2 * eps)
            assert abs(fd - g[name].reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), name


def test_adam_matches_torch():
    r = np.random.default_rng(4)
    p = {"a": r.normal(size=(3, 2)), "b": r.normal(size=5)}
    tp = [torch.tensor(p["a"], requires_grad=True), torch.tensor(p["b"], requires_grad=True)]
    opt = torch.optim.Adam(tp, lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    ad = CN.Adam(p, lr=1e-2)
    for step in range(5):
        g = {"a": r.normal(size=(3, 2)), "b": r.normal(size=5)}
        tp[0].grad = torch.tensor(g["a"])
        tp[1].grad = torch.tensor(g["b"])
        opt.step()
        p = ad.step(p, g)
    assert np.allclose(p["a"], tp[0].detach().numpy(), rtol=1e-12, atol=1e-14)
    assert np.allclose(p["b"], tp[1].detach().numpy(), rtol=1e-12, atol=1e-14)


def test_features_scatter_innovation():
    u = np.arange(16.0)[None, :]
    y = np.array([1.0, 2.0, 3.0, 4.0])
    x = CN.features(u, y, 0.5)
    assert np.allclose(x[0, 0], u[0])
    assert np.allclose(x[0, 1, ::4], (y - u[0, ::4]) / 0.5)
    assert np.all(x[0, 1, 1::4] == 0)
    # an unobserved point (NaN) has innovation zero
    ym = y.copy()
    ym[2:] = np.nan
    xm = CN.features(u, ym, 0.5)
    assert np.allclose(xm[0, 1, 0:8:4], (y[:2] - u[0, 0:8:4]) / 0.5)
    assert np.all(xm[0, 1, 8::4] == 0) and np.all(np.isfinite(xm))


def test_bf16_rounding_of_the_oracle():
    # bf16_round keeps 8 significant bits, rounding to nearest with ties to even, like a
    # BF16 conversion of an FP32 value: exact on BF16 values, ties go to the even neighbour
    a = np.array([1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20,
                  -2.5, 0.0, 3.0 * 2.0 ** -130])
    want = np.array([1.0, 1.0 + 2.0 ** -7, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -2.5, 0.0, 3.0 * 2.0 ** -130])
    assert np.array_equal(CN.bf16_round(a), want)
    r = np.random.default_rng(0).normal(size=1000)
    d = np.abs(CN.bf16_round(r) - r) / np.abs(r)
    assert d.max() <= 2.0 ** -8 + 1e-12
    # the BF16-operand network agrees with the FP64 one to BF16 precision in its forward pass
    p = CN.init_params(8, 4, 3, 64, 1)
    x0 = np.random.default_rng(1).normal(size=(3, 2, 64))
    a64, _ = CN.forward(p, x0, 4, 3)
    a16, _ = CN.forward(p, x0, 4, 3, operands="bf16")
    assert 0 < np.max(np.abs(a16 - a64)) <= 2e-2 * np.max(np.abs(a64))
