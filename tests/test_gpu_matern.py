"""GPU parity of the Matern SALT noise (Eq. noise_solve2) against the FP64 oracle.

The window and jitter kernels with one Brownian motion per cell and three
chained P1 solves per step.  Tolerances as for the mode expansion: FP64 fields
1e-10 and FP32 fields 1e-4 relative to the oracle's max-norm after a window.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

from workloads import get_config, random_state, random_increments, random_drift, random_obs
from oracle import filter as OF
from oracle import rng as ORNG
from tests.helpers import assert_decisions, gpu_model, jitter_moves_vs_oracle, oracle_model, rel_err, tdev

pytestmark = pytest.mark.gpu


def _cfg(name):
    base, _, over = name.partition("@")
    cfg = get_config(base)
    for kv in filter(None, over.split(",")):
        key, val = kv.split("=")
        cfg = dataclasses.replace(cfg, **{key: type(getattr(cfg, key))(val)})
    return cfg


def _case(cfg, N, seed, Ns=None, lam=False):
    Ns = cfg.Ns if Ns is None else Ns
    om = oracle_model(cfg)
    u0 = random_state(cfg, N, seed)
    m0 = np.stack([om.m_from_u(u) for u in u0])
    dW = random_increments(cfg, N, seed + 1, steps=Ns)
    la = random_drift(cfg, N, seed + 2, steps=Ns, scale=0.3) if lam else None
    return om, m0, dW, la


@pytest.mark.parametrize("name,N", [("cfg1m_f64", 4), ("cfg1m_f64@n=1024,M=64,Ns=3", 2),
                                    ("cfg1m_f64@eta=1.0,kappa=2.0,matern_k=1", 3), ("cfg1m_f64@n=128", 3)])
@pytest.mark.parametrize("lam", [False, True])
def test_matern_window_f64(name, N, lam):
    cfg = _cfg(name)
    g = gpu_model(cfg)
    assert g.K == cfg.n and g.layout == "cta"
    om, m0, dW, la = _case(cfg, N, 11, lam=lam)
    ref = om.ensemble_window(m0, dW, la)
    y = random_obs(cfg, 3)
    out = g.ensemble_step(tdev(m0, g.dtype), tdev(dW, g.dtype), None if la is None else tdev(la, g.dtype),
                          y=tdev(y, g.dtype))
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    assert rel_err(out["m"].cpu().numpy(), ref[0]) < 1e-10
    assert rel_err(out["u"].cpu().numpy(), ref[1]) < 1e-10
    assert np.all(np.abs(out["iters"].cpu().numpy() - ref[2].sum(axis=1)) <= cfg.Ns)
    lg = OF.girsanov_logG(la, dW, cfg.dt) if la is not None else np.zeros(N)
    assert np.allclose(out["nll"].cpu().numpy(), OF.nll(ref[1], y, cfg.sigma), rtol=1e-9)
    assert np.allclose(out["logG"].cpu().numpy(), lg, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("name,N", [("cfg2m_f32", 3), ("cfg2m_f32@n=256,M=64", 4), ("cfg2m_f32@n=4096,M=128,Ns=4", 2)])
@pytest.mark.parametrize("layout", ["auto", "cta"])
def test_matern_window_f32(name, N, layout):
    # auto: one warp per particle at n = 256 and 1024, the CTA layout at n = 4096
    cfg = _cfg(name)
    g = gpu_model(cfg, layout=layout)
    assert g.layout == ("warp" if layout == "auto" and cfg.n <= 1024 else "cta")
    om, m0, dW, la = _case(cfg, N, 31, lam=True)
    ref = om.ensemble_window(m0, dW, la)
    out = g.ensemble_step(tdev(m0, g.dtype), tdev(dW, g.dtype), tdev(la, g.dtype))
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    assert rel_err(out["m"].cpu().numpy(), ref[0]) < 1e-4
    assert rel_err(out["u"].cpu().numpy(), ref[1]) < 1e-4


def test_matern_draw_increments_one_per_cell():
    cfg = get_config("cfg1m_f64")
    g = gpu_model(cfg)
    dW = g.draw_increments(3, cfg.Ns, 123, ORNG.TAG_PRIOR_DW, 9, particle0=2).cpu().numpy()
    ref = ORNG.window_increments(123, ORNG.TAG_PRIOR_DW, 3, cfg.Ns, cfg.n, cfg.dt, 9, particle0=2)
    assert dW.shape == (3, cfg.Ns, cfg.n)
    assert np.max(np.abs(dW - ref)) < 1e-13


def test_matern_f32_draws_philox4x32():
    # the FP32 Matern increments come from Philox4x32-10: the raw words equal the oracle's bit
    # for bit, so the normals agree to the FP32 Box-Muller transform's error (a few 1e-6
    # relative, 1e-5 absolute at |z| <= 6), across counters whose words exceed 32 bits
    cfg = get_config("cfg2m_f32")
    g = gpu_model(cfg)
    for seed, ctr, p0 in ((123, 9, 2), (2**40 + 7, 2**33 + 5, 1000)):
        dW = g.draw_increments(3, cfg.Ns, seed, ORNG.TAG_PRIOR_DW, ctr, particle0=p0).double().cpu().numpy()
        ref = ORNG.window_increments(seed, ORNG.TAG_PRIOR_DW, 3, cfg.Ns, cfg.n, cfg.dt, ctr, particle0=p0,
                                     gen=ORNG.GEN32)
        other = ORNG.window_increments(seed, ORNG.TAG_PRIOR_DW, 3, cfg.Ns, cfg.n, cfg.dt, ctr, particle0=p0)
        z, zr = dW / np.sqrt(cfg.dt), ref / np.sqrt(cfg.dt)
        assert np.max(np.abs(z - zr)) < 1e-5
        assert np.max(np.abs(z - zr) / np.maximum(1.0, np.abs(zr))) < 1e-5
        assert np.max(np.abs(dW - other)) > 0.1   # not the 4x64 stream


@pytest.mark.parametrize("lam", [False, True])
def test_matern_jitter_matches_oracle(lam):
    cfg = get_config("cfg1m_f64")
    g = gpu_model(cfg)
    om = oracle_model(cfg)
    N, theta = 6, 0.6
    m0 = np.stack([om.m_from_u(u) for u in random_state(cfg, N, 50)])
    dW = random_increments(cfg, N, 51)
    la = random_drift(cfg, N, 52, scale=0.2) if lam else None
    y = random_obs(cfg, 53)
    n_iter, seed, ctr = 3, 77, 1000
    ref = OF.jitter(om, m0, dW, la, y, cfg.sigma, theta, cfg.rho, n_iter, seed, ctr)
    dt = g.dtype
    m0d, dWd, yd = tdev(m0, dt), tdev(dW, dt), tdev(y, dt)
    lad = None if la is None else tdev(la, dt)
    st = g.ensemble_step(m0d, dWd, lad, yd)
    nll, logG, m_end, u_end = st["nll"], st["logG"], st["m"], st["u"]
    acc, _, status = g.jitter(m0d, dWd, lad, yd, nll, logG, m_end, u_end, theta, cfg.rho, n_iter, seed, ctr)
    torch.cuda.synchronize()
    assert np.all(status.cpu().numpy() == 0)
    acc_g = acc.cpu().numpy()
    assert np.array_equal(acc_g, ref[5])
    assert 0 < ref[5].sum() < N * n_iter
    assert rel_err(dWd.cpu().numpy(), ref[0]) < 1e-10
    assert rel_err(u_end.cpu().numpy(), ref[4]) < 1e-10
    assert np.allclose(nll.cpu().numpy(), ref[1], rtol=1e-9)


@pytest.mark.parametrize("name,lam,layout", [("cfg2m_f32", False, "warp"), ("cfg2m_f32", True, "cta"),
                                             ("cfg2m_f32@n=256,M=64", True, "warp")])
def test_matern_jitter_f32_matches_oracle(name, lam, layout):
    # the FP32 Matern jitter kernels of both layouts against the FP64 oracle, move by move from
    # the GPU's state: decisions equal unless the oracle's margin is within what the FP32 field
    # tolerance allows, noise and fields of moves both accept to FP32 tolerance (rho = 0.5 and
    # theta = 1, so that the chains both accept and reject)
    cfg = _cfg(name)
    g = gpu_model(cfg, layout=layout)
    assert g.layout == layout
    om = oracle_model(cfg)
    N, theta, rho = 3, 1.0, 0.5
    m0 = np.stack([om.m_from_u(u) for u in random_state(cfg, N, 50)])
    dW = random_increments(cfg, N, 51)
    la = random_drift(cfg, N, 52, scale=0.2) if lam else None
    y = random_obs(cfg, 53)
    dt = g.dtype
    recs = jitter_moves_vs_oracle(g, om, cfg, tdev(m0, dt), tdev(dW, dt), None if la is None else tdev(la, dt),
                                  tdev(y, dt), theta, 4, 77, 1000, range(N), 1e-4, rho=rho)
    assert_decisions(recs, exact=False)
    assert 0 < sum(r[3] for r in recs) < len(recs)


def test_matern_cycle_matches_oracle():
    # a whole assimilation cycle (tempering, resampling, jittering) with the Matern noise
    from paper_2402_06927_gb300.filter import EnsembleFilter
    cfg = get_config("cfg1m_f64", N=16, n_jitter=2)
    g = gpu_model(cfg)
    om = oracle_model(cfg)
    N = cfg.N
    m0 = np.stack([om.m_from_u(u) for u in random_state(cfg, N, 70, scale=0.1)])
    y = random_obs(cfg, 71)
    seed, cycle = 9, 2
    dW = ORNG.window_increments(seed, ORNG.TAG_PRIOR_DW, N, cfg.Ns, cfg.n, cfg.dt, cycle)
    ref = OF.assimilation_cycle(om, m0, y, cfg.sigma, cfg.ess_min, cfg.rho, cfg.n_jitter, seed, cycle, dW=dW)
    f = EnsembleFilter(g, N, cfg.Ns, cfg.ess_min, cfg.rho, cfg.n_jitter, seed)
    f.set_state(tdev(m0, g.dtype))
    st = f.cycle(tdev(y, g.dtype), cycle)
    assert len(st.stages) == len(ref["stages"]) >= 2
    for a, b in zip(st.stages, ref["stages"]):
        assert abs(a.dtheta - b["dtheta"]) <= 1e-9 * b["dtheta"]
    assert rel_err(f.u_end.cpu().numpy(), ref["u_end"]) < 1e-8
    assert rel_err(f.dW.cpu().numpy(), ref["dW"]) < 1e-8


def test_matern_full_size_sampled():
    # the Matern bench configuration (n = 1024, N = 1024, Ns = 10, FP32): every particle is
    # propagated in one launch, as the bench runs it, and three sampled particles are
    # recomputed by the oracle
    cfg = get_config("cfg2m_f32")
    g = gpu_model(cfg)
    assert g.layout == "warp"
    N = cfg.N
    u0 = random_state(cfg, N, 41)
    m0 = g.m_from_u(tdev(u0, g.dtype))
    dW = g.draw_increments(N, cfg.Ns, 7, ORNG.TAG_PRIOR_DW, 0)
    y = random_obs(cfg, 4)
    out = g.ensemble_step(m0, dW, None, tdev(y, g.dtype))
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    om = oracle_model(cfg)
    dWh = dW.double().cpu().numpy()
    m0h = m0.double().cpu().numpy()
    for p in (0, 517, N - 1):
        mref, uref, _, ok = om.window(m0h[p], dWh[p])
        assert ok
        assert rel_err(out["m"][p].cpu().numpy(), mref) < 1e-4
        assert rel_err(out["u"][p].cpu().numpy(), uref) < 1e-4
        assert abs(out["nll"][p].item() - OF.nll(uref[None], y, cfg.sigma)[0]) < 1e-3 * max(1.0, out["nll"][p].item())


def test_matern_layouts_agree_at_full_ensemble_size():
    # the warp-per-particle and CTA Matern kernels on the same 1024-particle window and
    # jitter call: equal to FP32 rounding, with the same jitter decisions
    cfg = get_config("cfg2m_f32")
    gw, gc = gpu_model(cfg, layout="warp"), gpu_model(cfg, layout="cta")
    assert gw.layout == "warp" and gc.layout == "cta"
    N = cfg.N
    u0 = torch.tensor(random_state(cfg, 1, 3)[0], dtype=torch.float32, device="cuda")
    m0, _ = gw.prior_sample(N, u0, 5, 0.05)
    dW = gw.draw_increments(N, cfg.Ns, 9, ORNG.TAG_PRIOR_DW, 0)
    lam = torch.tensor(random_drift(cfg, N, 6, scale=0.2), dtype=torch.float32, device="cuda")
    y = gw.synth_obs(u0, 2, 1)
    outs = []
    for g in (gw, gc):
        d = dW.clone()
        st = g.ensemble_step(m0, d, lam, y)
        acc, _, status = g.jitter(m0, d, lam, y, st["nll"], st["logG"], st["m"], st["u"], 0.5, cfg.rho, 3, 11, 7)
        torch.cuda.synchronize()
        assert torch.all(st["status"] == 0) and torch.all(status == 0)
        outs.append((st, acc, d))
    (a, acc_a, d_a), (b, acc_b, d_b) = outs
    scale = b["u"].abs().max().item()
    assert (a["u"] - b["u"]).abs().max().item() < 1e-4 * scale
    assert (acc_a != acc_b).float().mean().item() < 0.02     # decisions differ only at coin flips
    same = acc_a == acc_b
    assert (d_a[same] - d_b[same]).abs().max().item() < 1e-4


@pytest.mark.parametrize("ckpt", [2, None])
def test_matern_adjoint_matches_oracle_tangent_linear(ckpt):
    # the reverse-mode adjoint through the Matern noise map (its transpose: k solves per
    # step) against the oracle's tangent-linear gradient over all n drifts of every step;
    # ckpt = 2 recomputes the second segment, None keeps every forward state
    from oracle import nudge as ON
    cfg = get_config("cfg1m_f64")
    g = gpu_model(cfg)
    om, m0, dW, la = _case(cfg, 2, 61, Ns=3, lam=True)
    la = 0.2 * la / 0.3
    y = random_obs(cfg, 64)
    out = g.adjoint_window(tdev(m0, g.dtype), tdev(dW, g.dtype), tdev(la, g.dtype), tdev(y, g.dtype), ckpt=ckpt)
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    for p in range(2):
        J, grad = ON.cost_and_gradient(om, m0[p], dW[p], la[p], y, cfg.sigma)
        assert abs(out["J"][p].item() - J) <= 1e-10 * J
        assert rel_err(out["g_lam"][p].cpu().numpy(), grad) < 1e-8
        assert rel_err(out["g_dW"][p].cpu().numpy(), (grad - cfg.dt * la[p]) / cfg.dt) < 1e-8


def test_matern_mala_matches_oracle():
    # MALA on the Matern noise (n drifts per step), gradients from the adjoint: the oracle's
    # keyed decisions and noise
    cfg = get_config("cfg1m_f64")
    g = gpu_model(cfg)
    om, m0, dW, la = _case(cfg, 2, 31, Ns=3, lam=True)
    la = 0.2 * la / 0.3
    y = random_obs(cfg, 34)
    theta, h, n_iter, seed, ctr = 0.7, 0.25, 3, 5, 40
    ref_dW, ref_nll, ref_lg, ref_acc = OF.mala_jitter(om, m0, dW, la, y, cfg.sigma, theta, h, n_iter, seed, ctr)
    dWd = tdev(dW, g.dtype)
    out = g.mala_jitter(tdev(m0, g.dtype), dWd, tdev(la, g.dtype), tdev(y, g.dtype), theta, h, n_iter, seed, ctr,
                        ckpt=2)
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    assert np.array_equal(out["accepts"].cpu().numpy(), ref_acc)
    assert 0 < ref_acc.sum() < 2 * n_iter
    assert rel_err(dWd.cpu().numpy(), ref_dW) < 1e-8
    assert np.allclose(out["nll"].cpu().numpy(), ref_nll, rtol=1e-8)
    assert np.allclose(out["logG"].cpu().numpy(), ref_lg, rtol=1e-8, atol=1e-12)


def _matern_nudge_case():
    cfg = get_config("cfg1m_f64", n=128, M=16, Ns=3)
    om = oracle_model(cfg)
    u0 = random_state(cfg, 2, 11)
    m0 = np.stack([om.m_from_u(u) for u in u0])
    y = random_obs(cfg, 12)
    return cfg, om, m0, y


def test_matern_nudge_open_loop_matches_oracle():
    # L-BFGS over one drift per cell and step (Lambda in Q_h), the optimiser's vectors in the
    # workspace: the oracle's minimiser (scipy L-BFGS-B on the tangent-linear gradient)
    from oracle import nudge as ON
    cfg, om, m0, y = _matern_nudge_case()
    g = gpu_model(cfg)
    out = g.nudge(tdev(m0, g.dtype), tdev(y, g.dtype), cfg.Ns, mode="open_loop", max_iter=200, gtol=1e-10,
                  ckpt=2, seed=4, ctr=1)
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    lam = out["lam"].cpu().numpy()
    assert lam.shape == (2, cfg.Ns, cfg.n)
    for p in range(2):
        ref, res = ON.nudge_open_loop(om, m0[p], y, cfg.sigma, cfg.Ns, cfg.Q, gtol=1e-12)
        assert rel_err(lam[p], ref) < 1e-5
        assert abs(out["J"][p].item() - res.fun) <= 1e-9 * res.fun
        z = ORNG.normals(4, ORNG.TAG_NUDGE, cfg.Q, np.arange(cfg.Ns, dtype=np.uint64), np.uint64(p), np.uint64(1))
        assert np.allclose(out["dW"][p].cpu().numpy(), math.sqrt(cfg.dt) * z, rtol=1e-13, atol=1e-15)


def test_matern_nudge_sequential_matches_oracle():
    from oracle import nudge as ON
    cfg, om, m0, y = _matern_nudge_case()
    g = gpu_model(cfg)
    out = g.nudge(tdev(m0, g.dtype), tdev(y, g.dtype), cfg.Ns, mode="sequential", max_iter=100, gtol=1e-10,
                  ckpt=2, seed=3, ctr=7)
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    for p in range(2):
        lam, dW = ON.nudge_sequential(om, m0[p], y, cfg.sigma, cfg.Ns, cfg.Q, seed=3, particle=p, ctr=7,
                                      gtol=1e-12)
        assert np.allclose(out["dW"][p].cpu().numpy(), dW, rtol=1e-13, atol=1e-15)
        assert rel_err(out["lam"][p].cpu().numpy(), lam) < 1e-5
