"""GPU parity of the learned drift proposal network against its FP64 oracle.

FP32 kernels with FP32 accumulation: outputs within 1e-4 and parameter
gradients within 2e-4 of each tensor's largest entry; Adam within 1e-5.
BF16 operands with FP32 accumulation (the tensor-core path): outputs within 1e-2
of the largest output of the FP64 oracle (the precision stated for BF16
inference).  Its gradients differ from the FP64 oracle's by up to a fifth of a
tensor's largest entry (ReLU masks flip where a pre-activation lies within BF16
rounding of zero, and the backward signal passes through four layers of BF16
operands), so they are compared with the oracle evaluated with the same BF16
rounding of both operands of every contraction: outputs, loss and gradients
within 2e-3 of the largest entry (FP32 against FP64 accumulation, and the rare
operand that FP32 and FP64 values round to neighbouring BF16 values).
"""
import numpy as np
import pytest
import torch

from oracle import convnet as CN
from tests.helpers import require_lib

pytestmark = pytest.mark.gpu


def _flat(p):
    keys = [f"w{l}" for l in range(4)]
    out = []
    for l in range(4):
        out += [p[f"w{l}"].ravel(), p[f"b{l}"].ravel()]
    out += [p["wh"].ravel(), p["bh"].ravel()]
    return np.concatenate(out)


def _unflat(v, p):
    out, o = {}, 0
    for k in [f"w0", "b0", "w1", "b1", "w2", "b2", "w3", "b3", "wh", "bh"]:
        out[k] = v[o:o + p[k].size].reshape(p[k].shape)
        o += p[k].size
    return out


def _case(n=256, K=4, Ns=3, C=16, M=32, B=6, seed=0):
    r = np.random.default_rng(seed)
    p = CN.init_params(C, K, Ns, n, seed)
    for l in range(4):
        p[f"b{l}"] = 0.05 * r.normal(size=C)
    p["bh"] = 0.05 * r.normal(size=K * Ns)
    x = np.arange(n) * 40.0 / n
    u = 0.2 / np.cosh(x - 27)[None, :] + 0.1 * r.normal(size=(B, 1)) * np.sin(2 * np.pi * x / 40)[None, :]
    y = r.normal(scale=0.1, size=(B, M)) + u[:, :: n // M]
    target = r.normal(scale=0.5, size=(B, Ns, K))
    return p, u, y, target


@pytest.mark.parametrize("masked", [False, True])
def test_forward_and_gradients_match_oracle(masked):
    api = require_lib()
    n, K, Ns, C, M, sigma = 256, 4, 3, 16, 32, 0.05
    p, u, y, target = _case(n, K, Ns, C, M)
    if masked:   # unobserved points (NaN) carry zero innovation
        y[:, M // 2 + 1:] = np.nan
    net = api.ProposalNet(n, K, Ns, M, sigma, C=C, params=torch.tensor(_flat(p), dtype=torch.float32))
    ud = torch.tensor(u, dtype=torch.float32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    lam = net.forward(ud, yd).cpu().numpy()
    x0 = np.stack([CN.features(u[b:b + 1], y[b], sigma)[0] for b in range(u.shape[0])])
    ref, _ = CN.forward(p, x0, K, Ns)
    assert np.max(np.abs(lam - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))
    loss, grads = net.loss_and_grad(ud, yd, torch.tensor(target, dtype=torch.float32, device="cuda"))
    L, g = CN.loss_and_grad(p, x0, target, K, Ns)
    assert abs(loss.item() - L) <= 1e-4 * L
    gg = _unflat(grads.cpu().numpy().astype(np.float64), p)
    for k in g:
        assert np.max(np.abs(gg[k] - g[k])) <= 2e-4 * max(1e-6, np.max(np.abs(g[k]))), k
    # shared observation vector (y stride 0) equals a broadcast batch
    lam_shared = net.forward(ud, yd[0].contiguous()).cpu().numpy()
    lam_bcast = net.forward(ud, yd[0:1].expand(u.shape[0], M).contiguous()).cpu().numpy()
    assert np.array_equal(lam_shared, lam_bcast)
    assert np.all(np.isfinite(lam))


def test_split_k_gradients_match_oracle_and_are_reproducible():
    # B = 600: every weight gradient (the head's over the batch, the convolutions' over
    # batch x positions) is split over k-chunks that are summed in a fixed order, so a
    # second evaluation gives the same bits
    api = require_lib()
    n, K, Ns, C, M, sigma = 256, 4, 3, 16, 32, 0.05
    p, u, y, target = _case(n, K, Ns, C, M, B=600, seed=3)
    net = api.ProposalNet(n, K, Ns, M, sigma, C=C, params=torch.tensor(_flat(p), dtype=torch.float32))
    ud = torch.tensor(u, dtype=torch.float32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    td = torch.tensor(target, dtype=torch.float32, device="cuda")
    _, g1 = net.loss_and_grad(ud, yd, td)
    g1 = g1.cpu().numpy()
    _, g2 = net.loss_and_grad(ud, yd, td)
    assert np.array_equal(g1, g2.cpu().numpy())
    x0 = np.stack([CN.features(u[b:b + 1], y[b], sigma)[0] for b in range(u.shape[0])])
    _, g = CN.loss_and_grad(p, x0, target, K, Ns)
    gg = _unflat(g1.astype(np.float64), p)
    for k in g:
        assert np.max(np.abs(gg[k] - g[k])) <= 2e-4 * max(1e-6, np.max(np.abs(g[k]))), k


def test_adam_matches_oracle():
    api = require_lib()
    n, K, Ns, C, M, sigma = 128, 2, 2, 8, 16, 0.05
    p, u, y, target = _case(n, K, Ns, C, M, B=4, seed=1)
    net = api.ProposalNet(n, K, Ns, M, sigma, C=C, params=torch.tensor(_flat(p), dtype=torch.float32))
    ad = CN.Adam({k: v.copy() for k, v in p.items()}, lr=1e-3)
    pref = {k: v.copy() for k, v in p.items()}
    r = np.random.default_rng(2)
    for step in range(3):
        gflat = r.normal(size=net.count).astype(np.float32)
        net.adam_step(torch.tensor(gflat, device="cuda"), lr=1e-3)
        pref = ad.step(pref, _unflat(gflat.astype(np.float64), p))
    got = net.params.cpu().numpy()
    assert np.max(np.abs(got - _flat(pref))) <= 1e-5


def test_training_reduces_the_loss():
    api = require_lib()
    n, K, Ns, C, M, sigma = 256, 4, 3, 16, 32, 0.05
    p, u, y, target = _case(n, K, Ns, C, M, B=64, seed=3)
    net = api.ProposalNet(n, K, Ns, M, sigma, C=C, seed=4)
    ud = torch.tensor(u, dtype=torch.float32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    td = torch.tensor(target, dtype=torch.float32, device="cuda")
    first = net.train_step(ud, yd, td, lr=3e-3).item()
    for _ in range(200):
        last = net.train_step(ud, yd, td, lr=3e-3).item()
    assert last < 0.5 * first


@pytest.mark.parametrize("shape", [(256, 4, 3, 16, 32, 6), (1024, 16, 20, 64, 64, 3)])
def test_bf16_forward_and_gradients_match_oracle(shape):
    # the tensor-core path at a small shape and at the shape the bench and the learned nudging
    # run (n = 1024, K = 16, Ns = 20, C = 64, M = 64), against the FP64 oracle network
    api = require_lib()
    n, K, Ns, C, M, B = shape
    sigma = 0.05
    p, u, y, target = _case(n, K, Ns, C, M, B=B, seed=7)
    net = api.ProposalNet(n, K, Ns, M, sigma, C=C, params=torch.tensor(_flat(p), dtype=torch.float32),
                          precision="bf16")
    ud = torch.tensor(u, dtype=torch.float32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    td = torch.tensor(target, dtype=torch.float32, device="cuda")
    lam = net.forward(ud, yd).cpu().numpy()
    x0 = np.stack([CN.features(u[b:b + 1], y[b], sigma)[0] for b in range(B)])
    ref, _ = CN.forward(p, x0, K, Ns)
    assert np.max(np.abs(lam - ref)) <= 1e-2 * np.max(np.abs(ref))
    ref_b, _ = CN.forward(p, x0, K, Ns, operands="bf16")
    assert np.max(np.abs(lam - ref_b)) <= 2e-3 * np.max(np.abs(ref_b))
    loss, grads = net.loss_and_grad(ud, yd, td)
    L, g = CN.loss_and_grad(p, x0, target, K, Ns, operands="bf16")
    assert abs(loss.item() - L) <= 2e-3 * L
    gg = _unflat(grads.cpu().numpy().astype(np.float64), p)
    for k in g:
        assert np.max(np.abs(gg[k] - g[k])) <= 2e-3 * max(1e-6, np.max(np.abs(g[k]))), k
    if n == 1024:
        # the FP32 path at the bench shape too
        net.set_precision("fp32")
        lam32 = net.forward(ud, yd).cpu().numpy()
        assert np.max(np.abs(lam32 - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))
        _, g32 = net.loss_and_grad(ud, yd, td)
        _, g64 = CN.loss_and_grad(p, x0, target, K, Ns)
        gg = _unflat(g32.cpu().numpy().astype(np.float64), p)
        for k in g64:
            assert np.max(np.abs(gg[k] - g64[k])) <= 2e-4 * max(1e-6, np.max(np.abs(g64[k]))), k


def test_bf16_training_reduces_the_loss():
    api = require_lib()
    n, K, Ns, C, M, sigma = 256, 4, 3, 16, 32, 0.05
    p, u, y, target = _case(n, K, Ns, C, M, B=64, seed=3)
    net = api.ProposalNet(n, K, Ns, M, sigma, C=C, seed=4, precision="bf16")
    ud = torch.tensor(u, dtype=torch.float32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    td = torch.tensor(target, dtype=torch.float32, device="cuda")
    first = net.train_step(ud, yd, td, lr=3e-3).item()
    for _ in range(200):
        last = net.train_step(ud, yd, td, lr=3e-3).item()
    assert last < 0.5 * first
