"""GPU parity of the SCH model kernels against the FP64 oracle (through the C ABI).

Tolerances (max-norm, relative to the oracle's max-norm):
* FP64 fields after one window: 1e-10 (the Picard iteration stops at 1e-13
  relative; the two sides differ only by rounding order).
* FP32 fields after one window: 1e-4 (single-precision rounding over
  Ns implicit solves with tolerance 1e-6).
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

from workloads import get_config, random_state, random_increments, random_drift, random_obs, u0_profile
from oracle import filter as OF
from oracle import rng as ORNG
from tests.helpers import gpu_model, oracle_model, tdev, rel_err

pytestmark = pytest.mark.gpu

F64_TOL = 1e-10
F32_TOL = 1e-4


def _case(cfg, N, seed, Ns=None, lam=False):
    Ns = cfg.Ns if Ns is None else Ns
    om = oracle_model(cfg)
    u0 = random_state(cfg, N, seed)
    m0 = np.stack([om.m_from_u(u) for u in u0])
    dW = random_increments(cfg, N, seed + 1, steps=Ns)
    la = random_drift(cfg, N, seed + 2, steps=Ns) if lam else None
    return om, m0, dW, la


@pytest.mark.parametrize("name", ["cfg1_f64", "cfg3_f64", "cfg2_f32", "cfg5_f32"])
def test_helmholtz_both_ways(name):
    cfg = get_config(name)
    g = gpu_model(cfg)
    om = oracle_model(cfg)
    u = random_state(cfg, 3, 5)
    if cfg.dtype == "f32":
        u = u.astype(np.float32).astype(np.float64)
    ref_m = np.stack([om.m_from_u(v) for v in u])
    m = g.m_from_u(tdev(u, g.dtype)).cpu().numpy()
    if cfg.dtype == "f64":
        assert rel_err(m, ref_m) < F64_TOL
    else:
        # m = M^{-1} (M + alpha^2 K) u differentiates twice: the FP32 right-hand
        # side carries ~3 eps (4 alpha^2 / h) |u| of rounding and M^{-1} has norm
        # 3 / h, so |m - m_ref| <= 36 eps alpha^2 |u| / h^2 bounds the kernel's error
        eps = np.finfo(np.float32).eps
        bound = 36 * eps * cfg.alpha ** 2 * np.max(np.abs(u)) / cfg.h ** 2
        assert np.max(np.abs(m - ref_m)) <= bound
        assert np.max(np.abs(m - ref_m)) <= 1e-2 * np.max(np.abs(ref_m))
    # u = H^{-1} M m smooths: well conditioned in both precisions
    uu = g.u_from_m(tdev(ref_m, g.dtype)).cpu().numpy()
    assert rel_err(uu, u) < (F64_TOL if cfg.dtype == "f64" else F32_TOL)


@pytest.mark.parametrize("lam", [False, True])
def test_window_f64_cfg1(lam):
    cfg = get_config("cfg1_f64")
    g = gpu_model(cfg)
    om, m0, dW, la = _case(cfg, 6, 11, lam=lam)
    ref = om.ensemble_window(m0, dW, la)
    y = random_obs(cfg, 3)
    out = g.ensemble_step(tdev(m0, g.dtype), tdev(dW, g.dtype), None if la is None else tdev(la, g.dtype),
                          y=tdev(y, g.dtype))
    torch.cuda.synchronize()
    assert rel_err(out["m"].cpu().numpy(), ref[0]) < F64_TOL
    assert rel_err(out["u"].cpu().numpy(), ref[1]) < F64_TOL
    assert np.all(out["status"].cpu().numpy() == 0)
    # Picard counts follow the same stopping rule
    assert np.all(np.abs(out["iters"].cpu().numpy() - ref[2].sum(axis=1)) <= cfg.Ns)
    nll = OF.nll(ref[1], y, cfg.sigma)
    lg = OF.girsanov_logG(la, dW, cfg.dt) if la is not None else np.zeros(6)
    assert np.allclose(out["nll"].cpu().numpy(), nll, rtol=1e-9)
    assert np.allclose(out["logG"].cpu().numpy(), lg, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("solver,name", [("ea", "cfg1_f64"), ("ea", "cfg3_f64"), ("li", "cfg2_f32")])
def test_window_other_solver(solver, name):
    # each precision also runs the other Picard iteration; both reach the fixed point of Eq. fde1
    cfg = get_config(name)
    g = gpu_model(cfg, solver=solver)
    om, m0, dW, la = _case(cfg, 3, 13, Ns=4, lam=True)
    om.scheme = solver
    ref = om.ensemble_window(m0, dW, la)
    out = g.ensemble_step(tdev(m0, g.dtype), tdev(dW, g.dtype), tdev(la, g.dtype))
    torch.cuda.synchronize()
    tol = F64_TOL if cfg.dtype == "f64" else F32_TOL
    assert rel_err(out["m"].cpu().numpy(), ref[0]) < tol
    assert rel_err(out["u"].cpu().numpy(), ref[1]) < tol
    assert np.all(out["status"].cpu().numpy() == 0)
    if cfg.dtype == "f64":
        assert np.all(np.abs(out["iters"].cpu().numpy() - ref[2].sum(axis=1)) <= 4)


def test_window_f64_multiwarp():
    # n = 1024 in FP64: 256 threads per particle, exercises the cross-warp exchanges
    cfg = get_config("cfg3_f64")
    g = gpu_model(cfg)
    om, m0, dW, la = _case(cfg, 2, 21, Ns=4, lam=True)
    ref = om.ensemble_window(m0, dW, la)
    out = g.ensemble_step(tdev(m0, g.dtype), tdev(dW, g.dtype), tdev(la, g.dtype))
    torch.cuda.synchronize()
    assert rel_err(out["m"].cpu().numpy(), ref[0]) < F64_TOL
    assert rel_err(out["u"].cpu().numpy(), ref[1]) < F64_TOL


@pytest.mark.parametrize("name,N,layout", [("cfg2_f32", 3, "warp"), ("cfg2_f32", 3, "cta"), ("cfg5_f32", 2, "auto"),
                                           ("cfg2_f32@n=256", 3, "warp"), ("cfg2_f32@n=512", 4, "warp"),
                                           ("cfg2_f32@mu=2.0", 3, "warp"), ("cfg2_f32@mu=2.0", 2, "cta"),
                                           # the noise tables at their extremes: one harmonic, and 32
                                           # (K = 64, the largest K), with an odd harmonic count too
                                           ("cfg2_f32@K=2", 2, "warp"), ("cfg2_f32@K=64", 2, "warp"),
                                           ("cfg2_f32@K=6", 2, "warp"), ("cfg2_f32@K=64", 2, "cta")])
def test_window_f32(name, N, layout):
    # both kernel layouts against the oracle; the warp-per-particle kernels at
    # every sub-chunk length they are built for (n = 256, 512, 1024), and with a
    # viscosity large enough that the Picard matrix's reduced system is coupled
    # (at mu = 0.02 it is diagonal to 2^-30 and solved without the lane PCR)
    base, _, over = name.partition("@")
    cfg = get_config(base)
    if over:
        key, val = over.split("=")
        cfg = dataclasses.replace(cfg, **{key: type(getattr(cfg, key))(val)})
    g = gpu_model(cfg, layout=layout)
    om, m0, dW, la = _case(cfg, N, 31, lam=True)
    ref = om.ensemble_window(m0, dW, la)
    out = g.ensemble_step(tdev(m0, g.dtype), tdev(dW, g.dtype), tdev(la, g.dtype))
    torch.cuda.synchronize()
    assert rel_err(out["m"].cpu().numpy(), ref[0]) < F32_TOL
    assert rel_err(out["u"].cpu().numpy(), ref[1]) < F32_TOL
    assert np.all(out["status"].cpu().numpy() == 0)


@pytest.mark.parametrize("mu", [0.02, 2.0])
def test_window_f32_diagonal_helmholtz(mu):
    # at alpha = h / sqrt(6) the Helmholtz matrix's off-diagonal h/6 - alpha^2/h
    # vanishes, so its reduced system is diagonal too: with mu = 0.02 (Picard
    # reduced system diagonal) and mu = 2.0 (coupled) the warp kernels run their
    # other two reduced-solve specialisations
    cfg = get_config("cfg2_f32")
    cfg = dataclasses.replace(cfg, alpha=cfg.L / cfg.n / np.sqrt(6.0), mu=mu)
    g = gpu_model(cfg, layout="warp")
    om, m0, dW, la = _case(cfg, 3, 33, lam=True)
    ref = om.ensemble_window(m0, dW, la)
    out = g.ensemble_step(tdev(m0, g.dtype), tdev(dW, g.dtype), tdev(la, g.dtype))
    torch.cuda.synchronize()
    assert rel_err(out["m"].cpu().numpy(), ref[0]) < F32_TOL
    assert rel_err(out["u"].cpu().numpy(), ref[1]) < F32_TOL
    assert np.all(out["status"].cpu().numpy() == 0)


def test_window_full_size_sampled():
    # the bench configuration (n = 1024, N = 1024, Ns = 10, FP32): every particle
    # is propagated in the launch the bench times; three sampled particles are
    # recomputed by the oracle
    cfg = get_config("cfg2_f32")
    g = gpu_model(cfg)
    N = cfg.N
    u0 = random_state(cfg, N, 41)
    m0 = g.m_from_u(tdev(u0, g.dtype))
    dW = g.draw_increments(N, cfg.Ns, 7, 1, 0)
    y = random_obs(cfg, 4)
    out = g.ensemble_step(m0, dW, None, tdev(y, g.dtype))
    torch.cuda.synchronize()
    om = oracle_model(cfg)
    dWh = dW.double().cpu().numpy()
    m0h = m0.double().cpu().numpy()
    assert np.all(out["status"].cpu().numpy() == 0)
    for p in (0, 517, N - 1):
        mref, uref, _, ok = om.window(m0h[p], dWh[p])
        assert ok
        assert rel_err(out["m"][p].cpu().numpy(), mref) < F32_TOL
        assert rel_err(out["u"][p].cpu().numpy(), uref) < F32_TOL
        assert abs(out["nll"][p].item() - OF.nll(uref[None], y, cfg.sigma)[0]) < 1e-3 * max(1.0, out["nll"][p].item())


def test_draw_increments_match_oracle_generator():
    for name in ("cfg1_f64", "cfg2_f32"):
        cfg = get_config(name)
        g = gpu_model(cfg)
        dW = g.draw_increments(5, cfg.Ns, 123, ORNG.TAG_PRIOR_DW, 9, particle0=3).double().cpu().numpy()
        ref = ORNG.window_increments(123, ORNG.TAG_PRIOR_DW, 5, cfg.Ns, cfg.K, cfg.dt, 9, particle0=3)
        tol = 1e-13 if cfg.dtype == "f64" else 2e-6
        assert np.max(np.abs(dW - ref)) < tol * 5 * math.sqrt(cfg.dt)


def test_loglik_standalone():
    cfg = get_config("cfg1_f64")
    g = gpu_model(cfg)
    u = random_state(cfg, 7, 2)
    y = random_obs(cfg, 9)
    dW = random_increments(cfg, 7, 3)
    la = random_drift(cfg, 7, 4)
    nll, lg = g.loglik(tdev(u, g.dtype), tdev(y, g.dtype), tdev(dW, g.dtype), tdev(la, g.dtype))
    assert np.allclose(nll.cpu().numpy(), OF.nll(u, y, cfg.sigma), rtol=1e-12)
    assert np.allclose(lg.cpu().numpy(), OF.girsanov_logG(la, dW, cfg.dt), rtol=1e-12)
    nll0, lg0 = g.loglik(tdev(u, g.dtype), tdev(y, g.dtype))
    assert np.all(lg0.cpu().numpy() == 0.0)


def test_prior_sample_matches_oracle():
    cfg = get_config("cfg1_f64")
    g = gpu_model(cfg)
    om = oracle_model(cfg)
    ut = u0_profile(cfg)
    m_ref, u_ref = om.prior_sample(ut, 5, 4, 0.05)
    m, u = g.prior_sample(4, tdev(ut, g.dtype), 5, 0.05)
    assert rel_err(u.cpu().numpy(), u_ref) < 1e-11
    assert rel_err(m.cpu().numpy(), m_ref) < 1e-10


@pytest.mark.parametrize("name", ["exp1_f64", "cfg2m_f32"])
def test_prior_exp1_matches_oracle(name):
    # the Exp 1 initial ensemble (Eq. init_solve), members 3 .. 6 of a seeded draw
    cfg = get_config(name)
    g = gpu_model(cfg)
    om = oracle_model(cfg)
    m_ref, u_ref = om.prior_exp1(11, 4, particle0=3)
    m, u = g.prior_exp1(4, 11, particle0=3)
    tol = 1e-11 if cfg.dtype == "f64" else 1e-5
    assert rel_err(u.cpu().numpy(), u_ref) < tol
    # m = M^-1 (M + alpha^2 K) u amplifies the highest mesh mode by 1 + 12 alpha^2 / h^2
    # (about 7,900 at n = 1024): in FP32 the bound is a few float epsilons times that
    cond = 1 + 12 * cfg.alpha ** 2 / cfg.h ** 2
    mtol = 10 * tol if cfg.dtype == "f64" else 4 * 2.0 ** -24 * cond
    assert rel_err(m.cpu().numpy(), m_ref) < mtol
    assert np.all(u.cpu().numpy() >= 0.0)


def test_synth_obs_and_diagnostics():
    cfg = get_config("cfg1_f64")
    g = gpu_model(cfg)
    ut = u0_profile(cfg)
    y = g.synth_obs(tdev(ut, g.dtype), 3, 2).cpu().numpy()
    z = ORNG.normals(3, ORNG.TAG_OBS, cfg.M, np.uint64(0), np.uint64(0), np.uint64(2))
    assert np.allclose(y, ut[:: cfg.obs_stride] + cfg.sigma * z, rtol=1e-13, atol=1e-15)
    ens = random_state(cfg, 9, 8)
    d = g.diagnostics(tdev(ens, g.dtype), tdev(ut, g.dtype)).cpu().numpy()
    assert np.isclose(d[0], OF.emre(ut, ens), rtol=1e-12)
    assert np.isclose(d[1], OF.rb(ut, ens), rtol=1e-12)
    assert np.isclose(d[2], OF.res(ut, ens), rtol=1e-12)
    assert np.isclose(d[3], np.sqrt(np.mean((ens.mean(0) - ut) ** 2)), rtol=1e-12)


def test_nonfinite_input_reports_status():
    cfg = get_config("cfg1_f64")
    g = gpu_model(cfg)
    om, m0, dW, _ = _case(cfg, 3, 1)
    m0 = m0.copy()
    m0[1, 10] = np.nan
    out = g.ensemble_step(tdev(m0, g.dtype), tdev(dW, g.dtype))
    st = out["status"].cpu().numpy()
    assert st[1] & 2 and st[0] == 0 and st[2] == 0


def test_nonconvergence_reports_status():
    cfg = get_config("cfg1_f64", max_iter=1)
    g = gpu_model(cfg)
    om, m0, dW, _ = _case(cfg, 2, 1)
    out = g.ensemble_step(tdev(m0, g.dtype), tdev(dW, g.dtype))
    assert np.all(out["status"].cpu().numpy() & 1)


def test_empty_ensemble_is_noop():
    cfg = get_config("cfg1_f64")
    g = gpu_model(cfg)
    e = torch.empty((0, cfg.n), dtype=g.dtype, device="cuda")
    out = g.ensemble_step(e, torch.empty((0, cfg.Ns, cfg.K), dtype=g.dtype, device="cuda"))
    assert out["m"].shape == (0, cfg.n)


def test_layouts_agree_at_full_ensemble_size():
    # the two kernel layouts on the same 1024-particle window: equal to rounding,
    # with the same Picard iteration counts up to one per step
    cfg = get_config("cfg2_f32")
    gw, gc = gpu_model(cfg, layout="warp"), gpu_model(cfg, layout="cta")
    N = cfg.N
    u0 = torch.tensor(u0_profile(cfg), dtype=torch.float32, device="cuda")
    m0, _ = gw.prior_sample(N, u0, 5, 0.05)
    dW = gw.draw_increments(N, cfg.Ns, 9, 1, 0)
    y = gw.synth_obs(u0, 2, 1)
    a = gw.ensemble_step(m0, dW, None, y)
    b = gc.ensemble_step(m0, dW, None, y)
    torch.cuda.synchronize()
    scale = b["u"].abs().max().item()
    assert (a["u"] - b["u"]).abs().max().item() < F32_TOL * scale
    assert (a["m"] - b["m"]).abs().max().item() < F32_TOL * b["m"].abs().max().item()
    assert torch.all(a["status"] == 0) and torch.all(b["status"] == 0)
    assert (a["iters"] - b["iters"]).abs().max().item() <= cfg.Ns
    assert torch.allclose(a["nll"], b["nll"], rtol=1e-3)


@pytest.mark.parametrize("name,layout", [("cfg1_f64", "auto"), ("cfg2_f32", "warp"), ("cfg2_f32", "cta")])
def test_half_domain_observations(name, layout):
    # Exp 2: only the points of [0, L/2] are observed (NaN elsewhere); the fused window
    # likelihood and sch_loglik sum over the observed points only
    cfg = get_config(name)
    g = gpu_model(cfg, layout=layout)
    om, m0, dW, la = _case(cfg, 3, 61, lam=True)
    y = random_obs(cfg, 62, upto=0.5)
    assert np.isnan(y).sum() == cfg.M - (cfg.M // 2 + 1)
    ref = om.ensemble_window(m0, dW, la)
    out = g.ensemble_step(tdev(m0, g.dtype), tdev(dW, g.dtype), tdev(la, g.dtype), tdev(y, g.dtype))
    nll_ref = OF.nll(ref[1], y, cfg.sigma)
    tol = 1e-9 if cfg.dtype == "f64" else 1e-4
    assert np.allclose(out["nll"].cpu().numpy(), nll_ref, rtol=tol)
    yd = tdev(y, g.dtype)
    ll, _ = g.loglik(out["u"], yd)
    # the residuals are formed in the field precision, the sums in FP64
    tol_ll = 1e-9 if cfg.dtype == "f64" else 1e-6
    assert np.allclose(ll.cpu().numpy(), OF.nll(out["u"].double().cpu().numpy(), yd.double().cpu().numpy(),
                                                cfg.sigma), rtol=tol_ll)
    # the unobserved half carries no weight: the full-domain NLL is larger
    assert np.all(OF.nll(ref[1], random_obs(cfg, 62), cfg.sigma) > nll_ref)


@pytest.mark.parametrize("n,N", [(256, 9), (1024, 1024), (2048, 300), (4096, 1100)])
def test_diagnostics_f32(n, N):
    # float fields: the per-particle norms run in float (sums of at most n/32 squares a lane and
    # a 5-level warp tree: relative error below 133 2^-24, about 8e-6, at n = 4096; above 1024 the
    # truth and mean come from shared memory), the ensemble mean in double
    cfg = get_config("cfg2_f32", n=n, M=n // 16)
    g = gpu_model(cfg)
    ut = u0_profile(cfg).astype(np.float32).astype(np.float64)
    ens = random_state(cfg, N, 8).astype(np.float32).astype(np.float64)
    d = g.diagnostics(tdev(ens, g.dtype), tdev(ut, g.dtype)).cpu().numpy()
    assert np.isclose(d[0], OF.emre(ut, ens), rtol=1e-5)
    assert np.isclose(d[1], OF.rb(ut, ens), rtol=1e-9)
    assert np.isclose(d[2], OF.res(ut, ens), rtol=1e-5)
    assert np.isclose(d[3], np.sqrt(np.mean((ens.mean(0) - ut) ** 2)), rtol=1e-9)
