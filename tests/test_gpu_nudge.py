"""GPU parity of the adjoint and the nudging optimiser (through the C ABI).

* dJ/dlambda from the reverse-mode adjoint against the oracle's forward
  tangent-linear gradient (independent code) to 1e-8 relative, FP64;
* dJ/dlambda, dJ/ddW, dJ/dm0 against central finite differences of the GPU
  window cost on 16 random directions at the nudging workload size
  (n = 1024, 8 modes, 20-step window, every state kept as the bench runs it);
* gradients independent of the checkpoint interval;
* the L-BFGS drift of both schedules against the oracle's (scipy L-BFGS-B)
  minimiser, and the revealed increments bit-for-bit keyed draws;
* the torch.autograd.Function wrapper returns the adjoint's gradients;
* the FP32 adjoint, optimiser and MALA against the FP64 oracle (tolerances
  derived beside those tests).
"""
import math

import numpy as np
import pytest
import torch

from workloads import get_config, random_state, random_increments, random_drift, random_obs
from oracle import filter as OF
from oracle import nudge as ON
from oracle import rng as ORNG
from tests.helpers import assert_decisions, gpu_model, nll_error_bound, oracle_model, rel_err, tdev

pytestmark = pytest.mark.gpu


def _setup(cfg, N, seed, Ns=None, lam_scale=0.3):
    Ns = cfg.Ns if Ns is None else Ns
    om = oracle_model(cfg)
    u0 = random_state(cfg, N, seed)
    m0 = np.stack([om.m_from_u(u) for u in u0])
    dW = random_increments(cfg, N, seed + 1, steps=Ns)
    la = random_drift(cfg, N, seed + 2, scale=lam_scale, steps=Ns)
    y = random_obs(cfg, seed + 3)
    return om, m0, dW, la, y


@pytest.mark.parametrize("upto", [None, 0.5])
def test_adjoint_matches_oracle_tangent_linear(upto):
    cfg = get_config("cfg1_f64")
    g = gpu_model(cfg)
    om, m0, dW, la, y = _setup(cfg, 2, 5, Ns=4)
    if upto is not None:   # Exp 2: observations on [0, L/2] only
        y = random_obs(cfg, 8, upto=upto)
    out = g.adjoint_window(tdev(m0, g.dtype), tdev(dW, g.dtype), tdev(la, g.dtype), tdev(y, g.dtype), ckpt=2)
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    for p in range(2):
        J, grad = ON.cost_and_gradient(om, m0[p], dW[p], la[p], y, cfg.sigma)
        assert abs(out["J"][p].item() - J) <= 1e-10 * J
        assert rel_err(out["g_lam"][p].cpu().numpy(), grad) < 1e-8


@pytest.mark.parametrize("ck", [2, 3, 5, 7, None])
def test_adjoint_independent_of_checkpoint_interval(ck):
    # against every state recomputed from a checkpoint per step (ckpt = 1); at ckpt >= 5
    # (and None) the 5-step window is one segment whose states the forward pass keeps
    cfg = get_config("cfg1_f64")
    g = gpu_model(cfg)
    om, m0, dW, la, y = _setup(cfg, 2, 6, Ns=5)
    args = (tdev(m0, g.dtype), tdev(dW, g.dtype), tdev(la, g.dtype), tdev(y, g.dtype))
    ref = g.adjoint_window(*args, ckpt=1)
    out = g.adjoint_window(*args, ckpt=ck)
    for k in ("J", "g_lam", "g_dW", "g_m0"):
        assert torch.allclose(out[k], ref[k], rtol=1e-12, atol=1e-14), k


def test_adjoint_finite_differences_16_directions_nudging_workload():
    cfg = get_config("cfg3_f64")     # n = 1024, 8 modes, 20-step window, FP64
    g = gpu_model(cfg)
    N = 2
    om, m0, dW, la, y = _setup(cfg, N, 7, lam_scale=0.5)
    md, dWd, lad, yd = (tdev(a, g.dtype) for a in (m0, dW, la, y))
    out = g.adjoint_window(md, dWd, lad, yd)
    r = np.random.default_rng(8)

    def J(m, w, l):
        return g.adjoint_window(m, w, l, yd, want_dW=False, want_m0=False)["J"].cpu().numpy()

    for _ in range(16):
        dl = tdev(r.normal(size=la.shape), g.dtype)
        dw = tdev(r.normal(scale=math.sqrt(cfg.dt), size=dW.shape), g.dtype)
        dm = tdev(0.01 * r.normal(size=m0.shape), g.dtype)
        eps = 1e-6
        fd = (J(md + eps * dm, dWd + eps * dw, lad + eps * dl) - J(md - eps * dm, dWd - eps * dw, lad - eps * dl)) / (2 * eps)
        an = ((out["g_lam"] * dl).sum(dim=(1, 2)) + (out["g_dW"] * dw).sum(dim=(1, 2)) + (out["g_m0"] * dm).sum(dim=1))
        an = an.cpu().numpy()
        assert np.all(np.abs(fd - an) <= 1e-6 * np.maximum(1.0, np.abs(fd)))


def test_autograd_function_returns_adjoint_gradients():
    from paper_2402_06927_gb300.api import NudgingCost
    cfg = get_config("cfg1_f64")
    g = gpu_model(cfg)
    om, m0, dW, la, y = _setup(cfg, 3, 9, Ns=3)
    md, dWd, lad, yd = (tdev(a, g.dtype) for a in (m0, dW, la, y))
    lad.requires_grad_(True)
    dWd.requires_grad_(True)
    J = NudgingCost.apply(g, md, dWd, lad, yd, 2)
    (2.0 * J).sum().backward()
    ref = g.adjoint_window(md, dWd.detach(), lad.detach(), yd, ckpt=2)
    assert torch.allclose(lad.grad, 2.0 * ref["g_lam"], rtol=1e-13)
    assert torch.allclose(dWd.grad, 2.0 * ref["g_dW"], rtol=1e-13)


def _nudge_case():
    cfg = get_config("cfg1_f64", n=128, M=16, Ns=3)
    om = oracle_model(cfg)
    u0 = random_state(cfg, 2, 11)
    m0 = np.stack([om.m_from_u(u) for u in u0])
    y = random_obs(cfg, 12)
    return cfg, om, m0, y


@pytest.mark.slow
def test_nudge_open_loop_matches_oracle_at_the_nudging_workload_size():
    # pf_nudge at the full size of the nudging workload (n = 1024, K = 8, Ns = 20, FP64, L-BFGS
    # vectors in shared memory, every forward state kept) against the oracle's minimiser on one
    # particle; the drift within 1e-5 relative, the cost within 1e-9 relative
    cfg = get_config("cfg3_f64")
    g = gpu_model(cfg)
    om = oracle_model(cfg)
    m0 = np.stack([om.m_from_u(u) for u in random_state(cfg, 2, 11)])
    y = random_obs(cfg, 12)
    out = g.nudge(tdev(m0, g.dtype), tdev(y, g.dtype), cfg.Ns, mode="open_loop", max_iter=200, gtol=1e-10,
                  seed=4, ctr=1)
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    ref, res = ON.nudge_open_loop(om, m0[0], y, cfg.sigma, cfg.Ns, cfg.K, gtol=1e-12)
    assert rel_err(out["lam"][0].cpu().numpy(), ref) < 1e-5
    assert abs(out["J"][0].item() - res.fun) <= 1e-9 * res.fun


@pytest.mark.parametrize("ckpt", [2, None])
def test_nudge_open_loop_matches_oracle(ckpt):
    # ckpt = 2 recomputes each segment in the reverse sweep; None keeps the forward states
    cfg, om, m0, y = _nudge_case()
    g = gpu_model(cfg)
    out = g.nudge(tdev(m0, g.dtype), tdev(y, g.dtype), cfg.Ns, mode="open_loop", max_iter=200, gtol=1e-10,
                  ckpt=ckpt, seed=4, ctr=1)
    torch.cuda.synchronize()
    lam = out["lam"].cpu().numpy()
    for p in range(2):
        ref, res = ON.nudge_open_loop(om, m0[p], y, cfg.sigma, cfg.Ns, cfg.K, gtol=1e-12)
        assert rel_err(lam[p], ref) < 1e-5
        assert abs(out["J"][p].item() - res.fun) <= 1e-9 * res.fun
        z = ORNG.normals(4, ORNG.TAG_NUDGE, cfg.K, np.arange(cfg.Ns, dtype=np.uint64), np.uint64(p), np.uint64(1))
        assert np.allclose(out["dW"][p].cpu().numpy(), math.sqrt(cfg.dt) * z, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("ckpt", [2, None])
def test_nudge_sequential_matches_oracle(ckpt):
    cfg, om, m0, y = _nudge_case()
    g = gpu_model(cfg)
    out = g.nudge(tdev(m0, g.dtype), tdev(y, g.dtype), cfg.Ns, mode="sequential", max_iter=100, gtol=1e-10,
                  ckpt=ckpt, seed=3, ctr=7)
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    for p in range(2):
        lam, dW = ON.nudge_sequential(om, m0[p], y, cfg.sigma, cfg.Ns, cfg.K, seed=3, particle=p, ctr=7,
                                      gtol=1e-12)
        assert np.allclose(out["dW"][p].cpu().numpy(), dW, rtol=1e-13, atol=1e-15)
        assert rel_err(out["lam"][p].cpu().numpy(), lam) < 1e-5


@pytest.mark.parametrize("lam_on", [False, True])
def test_mala_jitter_matches_oracle(lam_on):
    # MALA with the gradient from the reverse-mode adjoint against the oracle's MALA
    # with the tangent-linear gradient: the same keyed normals and uniforms, so the
    # same decisions, and the same noise within the two gradients' agreement
    cfg = get_config("cfg1_f64")
    g = gpu_model(cfg)
    om, m0, dW, la, y = _setup(cfg, 3, 31, Ns=3, lam_scale=0.2)
    la = la if lam_on else None
    theta, h, n_iter, seed, ctr = 0.7, 0.8, 3, 5, 40   # h large enough that some moves are rejected
    ref_dW, ref_nll, ref_lg, ref_acc = OF.mala_jitter(om, m0, dW, la, y, cfg.sigma, theta, h, n_iter, seed, ctr)
    dWd = tdev(dW, g.dtype)
    out = g.mala_jitter(tdev(m0, g.dtype), dWd, None if la is None else tdev(la, g.dtype), tdev(y, g.dtype), theta,
                        h, n_iter, seed, ctr, ckpt=2)
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    assert np.array_equal(out["accepts"].cpu().numpy(), ref_acc)
    assert 0 < ref_acc.sum() < 3 * n_iter
    assert rel_err(dWd.cpu().numpy(), ref_dW) < 1e-8
    assert np.allclose(out["nll"].cpu().numpy(), ref_nll, rtol=1e-8)
    assert np.allclose(out["logG"].cpu().numpy(), ref_lg, rtol=1e-8, atol=1e-12)


# FP32 (explicit-advection Picard, the path the learned proposal's training pairs take).
# Tolerances: the FP32 Picard iteration stops at 1e-6 relative, which the window's
# sensitivity amplifies by about ten, so J within 2e-6 and gradients within 2e-5 relative
# of the FP64 oracle (measured: 8e-8 and 8e-7).  The optimiser stops on FP32 gradients,
# so its drift is held to 3e-4 of the oracle's minimiser (measured 4e-5); the revealed
# increments are FP32 normals, within 4e-6 of the FP64 transform, times sqrt(dt).
@pytest.mark.parametrize("n,M", [(256, 32), (1024, 64)])
@pytest.mark.parametrize("ckpt", [2, None])
def test_adjoint_f32_matches_oracle_tangent_linear(n, M, ckpt):
    cfg = get_config("cfg2_f32", n=n, M=M)
    g = gpu_model(cfg)
    om, m0, dW, la, y = _setup(cfg, 2, 5, Ns=4)
    out = g.adjoint_window(tdev(m0, g.dtype), tdev(dW, g.dtype), tdev(la, g.dtype), tdev(y, g.dtype), ckpt=ckpt)
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    for p in range(2):
        J, grad = ON.cost_and_gradient(om, m0[p], dW[p], la[p], y, cfg.sigma)
        assert abs(out["J"][p].item() - J) <= 2e-6 * J
        assert rel_err(out["g_lam"][p].double().cpu().numpy(), grad) < 2e-5
        assert rel_err(out["g_dW"][p].double().cpu().numpy(), (grad - cfg.dt * la[p]) / cfg.dt) < 2e-5


@pytest.mark.parametrize("mode", ["open_loop", "sequential"])
def test_nudge_f32_matches_oracle(mode):
    cfg = get_config("cfg2_f32", n=256, M=32, Ns=3)
    g = gpu_model(cfg)
    om = oracle_model(cfg)
    m0 = np.stack([om.m_from_u(u) for u in random_state(cfg, 2, 11)])
    y = random_obs(cfg, 12)
    seed, ctr = (4, 1) if mode == "open_loop" else (3, 7)
    out = g.nudge(tdev(m0, g.dtype), tdev(y, g.dtype), cfg.Ns, mode=mode, max_iter=200, gtol=1e-6, seed=seed,
                  ctr=ctr)
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    for p in range(2):
        if mode == "open_loop":
            lam, res = ON.nudge_open_loop(om, m0[p], y, cfg.sigma, cfg.Ns, cfg.K, gtol=1e-12)
            z = ORNG.normals(seed, ORNG.TAG_NUDGE, cfg.K, np.arange(cfg.Ns, dtype=np.uint64), np.uint64(p),
                             np.uint64(ctr))
            dW = math.sqrt(cfg.dt) * z
            assert abs(out["J"][p].item() - res.fun) <= 1e-5 * res.fun
        else:
            lam, dW = ON.nudge_sequential(om, m0[p], y, cfg.sigma, cfg.Ns, cfg.K, seed=seed, particle=p, ctr=ctr,
                                          gtol=1e-12)
        assert rel_err(out["lam"][p].double().cpu().numpy(), lam) < 3e-4
        assert np.max(np.abs(out["dW"][p].double().cpu().numpy() - dW)) < 4e-6 * math.sqrt(cfg.dt) * 6


@pytest.mark.parametrize("n,M", [(256, 32), (1024, 64)])
def test_mala_f32_matches_oracle(n, M):
    # FP32 MALA against the FP64 oracle, move by move from the GPU's state (a one-move call
    # keyed ctr + j is move j): decisions equal unless the oracle's margin log alpha - log u is
    # within the change the FP32 tolerances can cause (the NLL at both points through fields
    # within 1e-4, the gradient within the FP32 adjoint tolerance 2e-5 through the proposal and
    # both proposal densities); the noise of moves both accept to FP32 tolerance
    cfg = get_config("cfg2_f32", n=n, M=M)
    g = gpu_model(cfg)
    om, m0, dW, la, y = _setup(cfg, 3, 31, Ns=3, lam_scale=0.2)
    theta, h, n_iter, seed, ctr = 0.7, 0.8, 3, 5, 40
    dWd = tdev(dW, g.dtype)
    m0d, lad, yd = tdev(m0, g.dtype), tdev(la, g.dtype), tdev(y, g.dtype)
    m0h, lah, yh = m0d.double().cpu().numpy(), lad.double().cpu().numpy(), yd.double().cpu().numpy()
    tau, ftol = 2e-5, 1e-4
    recs = []
    for j in range(n_iter):
        before = dWd.double().cpu().numpy()
        out = g.mala_jitter(m0d, dWd, lad, yd, theta, h, 1, seed, ctr + j)
        torch.cuda.synchronize()
        assert np.all(out["status"].cpu().numpy() == 0)
        acc = out["accepts"].cpu().numpy()
        u_scale = out["u"].abs().max().item()
        for p in range(3):
            r = OF.mala_jitter(om, m0h[p:p + 1], before[p:p + 1], lah[p:p + 1], yh, cfg.sigma, theta, h, 1, seed,
                               ctr + j, particle0=p, margins=True)
            dW_o, acc_o, info = r[0], r[3], r[4][0][2]
            bound = (theta * (nll_error_bound(info["nll0"], M, u_scale, cfg.sigma, ftol)
                              + nll_error_bound(info["nll1"], M, u_scale, cfg.sigma, ftol))
                     + info["gp"] * 0.5 * h * cfg.dt * tau * info["g"]
                     + 0.5 * tau * (info["rf"] * info["g"] + info["rb"] * info["gp"]))
            recs.append((p, j, int(acc[p]), int(acc_o[0]), float(info["margin"]), float(bound)))
            if acc[p] == 1 and acc_o[0] == 1:
                assert rel_err(dWd[p].double().cpu().numpy(), dW_o[0]) < 1e-5
    assert_decisions(recs, exact=False)
    assert 0 < sum(r[3] for r in recs) < len(recs)