"""GPU parity of the filter kernels against the FP64 oracle (through the C ABI).

* tempering: dtheta, ESS and normalised weights within 1e-12 relative;
* resampling: offspring indices bit-exact given the oracle's weights;
* PCN jitter: every move of the sampled particles replayed by the oracle from the
  GPU's state; decisions identical in FP64, and in FP32 identical wherever the
  oracle's Metropolis margin |(w0 - w1) - log U| exceeds the change of w0 - w1 that
  fields within the FP32 window tolerance can cause; the new state of every move
  both sides accept within the window tolerance;
* a whole assimilation cycle in FP64: same number of tempering stages, the
  same temperatures and ensemble within 1e-8.
"""
import math

import dataclasses

import numpy as np
import pytest
import torch

from workloads import get_config, random_state, random_increments, random_drift, random_obs, random_logweights
from oracle import filter as OF
from oracle import rng as ORNG
from tests.helpers import (assert_decisions, gpu_model, jitter_moves_vs_oracle, oracle_model, require_lib, rel_err,
                           tdev)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,spread,theta", [(1, 1.0, 0.0), (7, 0.01, 0.0), (64, 5.0, 0.0), (1024, 30.0, 0.25),
                                            (1025, 30.0, 0.0), (1500, 10.0, 0.1), (8192, 80.0, 0.5),
                                            (16384, 5.0, 0.9)])
def test_temper_matches_oracle(N, spread, theta):
    # N <= 1024 runs the cluster on 128-thread CTAs (one particle a thread), larger N on 256
    api = require_lib()
    phi = random_logweights(N, N, spread)
    lg = np.random.default_rng(N).normal(size=N)
    ess_min = 0.5 * N
    nll = phi + lg
    w, out = api.pf_temper(tdev(nll, torch.float64), tdev(lg, torch.float64), theta, ess_min)
    out = out.cpu().numpy()
    d, wb, e = OF.temper(nll - lg, theta, ess_min)
    assert abs(out[0] - d) <= 1e-12 * max(d, 1e-300) + 1e-300
    assert abs(out[1] - e) <= 1e-12 * e
    assert np.allclose(w.cpu().numpy(), wb, rtol=1e-11, atol=1e-300)
    # the new temperature follows from the kernel's own dtheta by the stated rule
    exp_theta = 1.0 if out[0] >= 1.0 - theta else theta + out[0]
    assert out[2] == exp_theta
    # out[3]: ESS of the whole remaining step
    e_rest = OF.ess(-(1.0 - theta) * (nll - lg))
    assert abs(out[3] - e_rest) <= 1e-12 * e_rest


@pytest.mark.parametrize("N,spread,theta", [(7, 0.01, 0.0), (64, 5.0, 0.0), (1024, 30.0, 0.25), (8192, 80.0, 0.5)])
def test_temper_halving_matches_oracle(N, spread, theta):
    # the halving search tries exact dyadic points: dtheta equal to the oracle's unless an ESS
    # lies within rounding of the threshold (then the neighbouring point)
    api = require_lib()
    phi = random_logweights(N, N + 7, spread)
    w, out = api.pf_temper(tdev(phi, torch.float64), None, theta, 0.5 * N, mode="halving")
    out = out.cpu().numpy()
    d, wb, e = OF.temper(phi, theta, 0.5 * N, mode="halving")
    assert out[0] == d or out[0] in (2 * d, 0.5 * d)
    if out[0] == d:
        assert abs(out[1] - e) <= 1e-12 * e
        assert np.allclose(w.cpu().numpy(), wb, rtol=1e-11, atol=1e-300)


@pytest.mark.parametrize("N", [1, 2, 5, 100, 1024, 8192])
def test_resample_bit_exact_given_oracle_weights(N):
    api = require_lib()
    r = np.random.default_rng(N)
    for trial in range(3):
        w = r.gamma(0.3 + trial, size=N)
        w /= w.sum()
        seed, ctr = 1000 + trial, 17 * trial
        idx = api.pf_resample(tdev(w, torch.float64), seed, ctr).cpu().numpy()
        ref = OF.systematic_resample(w, OF.resample_offset(seed, ctr))
        assert np.array_equal(idx, ref)


def test_resample_degenerate_and_inplace():
    api = require_lib()
    N = 6
    w = np.array([0.0, 0.0, 1.0, 0.0, 0.0, 0.0])
    a = torch.arange(N * 4, dtype=torch.float32, device="cuda").reshape(N, 4)
    b = torch.arange(N * 8, dtype=torch.float64, device="cuda").reshape(N, 8)
    idx = api.pf_resample(tdev(w, torch.float64), 3, 4, arrays=[a, b]).cpu().numpy()
    assert np.array_equal(idx, np.full(N, 2))
    assert torch.all(a == torch.tensor([8, 9, 10, 11], dtype=torch.float32, device="cuda"))
    assert torch.all(b[:, 0] == 16)
    src = torch.randn(N, 3, dtype=torch.float64, device="cuda").contiguous()
    dst = torch.empty_like(src)
    perm = torch.tensor([5, 4, 3, 2, 1, 0], dtype=torch.int32, device="cuda")
    api.pf_gather_rows(perm, src, dst)
    assert torch.equal(dst, src.flip(0))


@pytest.mark.parametrize("name,theta,lam,layout,upto", [("cfg1_f64", 0.4, False, "auto", None),
                                                        ("cfg1_f64", 1.0, True, "auto", None),
                                                        ("cfg2_f32", 0.3, False, "warp", None),
                                                        ("cfg2_f32", 0.3, True, "cta", None),
                                                        ("cfg2_f32", 0.3, True, "group16", None),
                                                        ("cfg2_f32", 0.3, False, "warp", 0.5)])
def test_jitter_matches_oracle(name, theta, lam, layout, upto):
    # every move of every particle replayed by the oracle from the GPU's state: FP64 decisions
    # all equal; FP32 decisions may differ only where the oracle's Metropolis margin is within
    # the change of w0 - w1 that fields within the FP32 window tolerance can cause
    cfg = get_config(name)
    g = gpu_model(cfg, layout=layout)
    om = oracle_model(cfg)
    N = 8 if cfg.dtype == "f64" else 3
    u0 = random_state(cfg, N, 50)
    m0 = np.stack([om.m_from_u(u) for u in u0])
    dW = random_increments(cfg, N, 51)
    la = random_drift(cfg, N, 52, scale=0.2) if lam else None
    y = random_obs(cfg, 53, upto=upto)   # upto = 0.5: Exp 2's half-domain observations
    dt = g.dtype
    tol = 1e-10 if cfg.dtype == "f64" else 1e-4
    # rho 0.5 in FP32 (the workload's 0.9999 moves so little that every proposal is accepted),
    # so that both outcomes occur
    rho = cfg.rho if cfg.dtype == "f64" else 0.5
    recs = jitter_moves_vs_oracle(g, om, cfg, tdev(m0, dt), tdev(dW, dt), None if la is None else tdev(la, dt),
                                  tdev(y, dt), theta, 4, 77, 1000, range(N), tol, rho=rho)
    assert_decisions(recs, exact=cfg.dtype == "f64")
    assert len(recs) == 4 * N
    if upto is None:   # both outcomes occur (with half the observations every move is accepted)
        assert 0 < sum(r[2] for r in recs) < len(recs)


def test_jitter_moves_equal_one_call():
    # n_iter moves in one call are the n_iter single-move calls with counters ctr .. ctr + n_iter - 1
    cfg = get_config("cfg2_f32")
    g = gpu_model(cfg)
    om = oracle_model(cfg)
    N = 64
    m0 = tdev(np.stack([om.m_from_u(u) for u in random_state(cfg, N, 56)]), g.dtype)
    y = tdev(random_obs(cfg, 57), g.dtype)
    outs = []
    for split in (False, True):
        dW = tdev(random_increments(cfg, N, 58), g.dtype)
        st = g.ensemble_step(m0, dW, None, y)
        if split:
            acc = sum(g.jitter(m0, dW, None, y, st["nll"], st["logG"], st["m"], st["u"], 0.5, cfg.rho, 1, 3, 40 + j)[0]
                      for j in range(4))
        else:
            acc = g.jitter(m0, dW, None, y, st["nll"], st["logG"], st["m"], st["u"], 0.5, cfg.rho, 4, 3, 40)[0]
        outs.append((acc.clone(), dW.clone(), st["u"].clone(), st["nll"].clone()))
    torch.cuda.synchronize()
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)


def test_jitter_theta_zero_accepts_everything():
    cfg = get_config("cfg1_f64")
    g = gpu_model(cfg)
    om = oracle_model(cfg)
    N = 4
    m0 = np.stack([om.m_from_u(u) for u in random_state(cfg, N, 60)])
    dW = random_increments(cfg, N, 61)
    y = random_obs(cfg, 62)
    dt = g.dtype
    m0d, dWd, yd = tdev(m0, dt), tdev(dW, dt), tdev(y, dt)
    st = g.ensemble_step(m0d, dWd, None, yd)
    acc, _, _ = g.jitter(m0d, dWd, None, yd, st["nll"], st["logG"], st["m"], st["u"], 0.0, cfg.rho, 3, 5, 0)
    assert np.all(acc.cpu().numpy() == 3)


@pytest.mark.parametrize("eager,mode", [(3, "largest"), (0, "largest"), (1, "largest"), (3, "halving")])
def test_cycle_matches_oracle_f64(eager, mode):
    # eager = 3: stages enqueued as device-gated stages; 0: stage by stage; 1: one gated
    # stage, then the stage-by-stage fallback; halving: the paper's search read literally
    from paper_2402_06927_gb300.filter import EnsembleFilter
    cfg = get_config("cfg1_f64", N=16, n_jitter=2)
    g = gpu_model(cfg)
    om = oracle_model(cfg)
    N = cfg.N
    u0 = random_state(cfg, N, 70, scale=0.1)
    m0 = np.stack([om.m_from_u(u) for u in u0])
    y = random_obs(cfg, 71)
    seed, cycle = 9, 2
    dW = ORNG.window_increments(seed, ORNG.TAG_PRIOR_DW, N, cfg.Ns, cfg.K, cfg.dt, cycle)
    ref = OF.assimilation_cycle(om, m0, y, cfg.sigma, cfg.ess_min, cfg.rho, cfg.n_jitter, seed, cycle, dW=dW,
                                temper_mode=mode)
    f = EnsembleFilter(g, N, cfg.Ns, cfg.ess_min, cfg.rho, cfg.n_jitter, seed, temper_mode=mode,
                       eager_stages=eager)
    f.set_state(tdev(m0, g.dtype))
    st = f.cycle(tdev(y, g.dtype), cycle)
    assert len(st.stages) == len(ref["stages"])
    for a, b in zip(st.stages, ref["stages"]):
        assert abs(a.dtheta - b["dtheta"]) <= 1e-9 * b["dtheta"]
        assert abs(a.theta - b["theta"]) <= 1e-9
    assert rel_err(f.u_end.cpu().numpy(), ref["u_end"]) < 1e-8
    assert rel_err(f.dW.cpu().numpy(), ref["dW"]) < 1e-8


@pytest.mark.parametrize("nudged,name", [(False, "cfg2_f32"), (True, "cfg2_f32"), (False, "cfg5_f32@n=2048")])
def test_gated_stages_equal_stage_by_stage_fp32(nudged, name):
    # the same FP32 cycles with device-gated stages and stage by stage: the same kernels take
    # the same decisions, so every array and stage statistic is bit-identical; with a drift
    # the resampled drift rows are compared too.  At n = 2048 the warp-group layout runs with
    # warm-started proposals (the filter's jitter workspace, shared by both filters): still
    # bit-identical, since every call's warm starts depend on that call alone
    from paper_2402_06927_gb300.filter import EnsembleFilter
    from workloads import u0_profile
    base, _, over = name.partition("@")
    cfg = get_config(base)
    if over:
        key, val = over.split("=")
        cfg = dataclasses.replace(cfg, **{key: type(getattr(cfg, key))(val)})
    g = gpu_model(cfg)
    N = 256
    u0 = torch.tensor(u0_profile(cfg), dtype=torch.float32, device="cuda")
    m0, _ = g.prior_sample(N, u0, 4, cfg.prior_scale)
    fs = [EnsembleFilter(g, N, cfg.Ns, 0.5 * N, cfg.rho, 3, 11, eager_stages=e) for e in (3, 0)]
    assert all(f.warm_jitter == (g.layout == "group") for f in fs)
    for f in fs:
        f.set_state(m0)
    names = ("m_start", "m_end", "u_end", "dW", "nll", "logG") + (("lam",) if nudged else ())
    for c in range(3):
        y = g.synth_obs(u0, 20 + c, 1)
        if nudged:
            lam = torch.tensor(random_drift(cfg, N, 60 + c, scale=0.2), dtype=torch.float32, device="cuda")
            for f in fs:
                f.set_drift(lam)
        snaps = [[], []]
        sts = [f.cycle(y, c, post=lambda f=f, k=k: snaps[k].append(f.u_end.clone())) for k, f in enumerate(fs)]
        # the work a cycle's post hook enqueued last sees the final analysis
        for k, f in enumerate(fs):
            assert snaps[k] and torch.equal(snaps[k][-1], f.u_end)
        assert [(s.dtheta, s.ess, s.theta) for s in sts[0].stages] == [(s.dtheta, s.ess, s.theta) for s in sts[1].stages]
        assert sts[0].forward_steps == sts[1].forward_steps
        for name in names:
            assert torch.equal(getattr(fs[0], name), getattr(fs[1], name)), name
        for f in fs:
            f.advance()


@pytest.mark.parametrize("name", ["cfg2_f32", "cfg5_f32"])
def test_jitter_full_size_sampled(name):
    # the jitter in the bench's launch configuration (cfg2: n = 1024, N = 1024, K = 8, warp
    # layout; cfg5: n = 4096, N = 8192, K = 32, warp-group layout; Ns = 10, FP32), driven move by
    # move through the whole ensemble: three sampled particles replayed by the oracle with their
    # own Philox particle indices at every move
    cfg = get_config(name)
    g = gpu_model(cfg)
    assert g.layout == ("warp" if cfg.n <= 1024 else "group")
    om = oracle_model(cfg)
    N, theta, seed, ctr = cfg.N, 0.5, 77, 1000
    n_iter = 4 if cfg.n > 1024 else cfg.n_jitter
    u0 = torch.tensor(random_state(cfg, 1, 3)[0], dtype=torch.float32, device="cuda")
    m0, _ = g.prior_sample(N, u0, 5, cfg.prior_scale)
    dW = g.draw_increments(N, cfg.Ns, 9, ORNG.TAG_PRIOR_DW, 0)
    y = g.synth_obs(u0, 2, 1)
    recs = jitter_moves_vs_oracle(g, om, cfg, m0, dW, None, y, theta, n_iter, seed, ctr, (0, 517, N - 1), 1e-4)
    assert_decisions(recs, exact=False)
