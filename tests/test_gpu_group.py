"""GPU parity of the warp-group kernels (several warps per particle, n = 2048 and 4096,
FP32 fields, explicit-advection Picard) against the FP64 oracle, through the C ABI.

The warp-group layout completes each constant cyclic solve across the particle's warps
through shared memory (the 2W boundary values of the warps' lane-level systems); these
tests run it at both lane widths it is built for (32 and 16 nodes a lane), with the
Picard matrix's reduced system coupled (mu = 0.02 at n >= 2048, and mu = 2) and with a
drift, and compare it with the one-CTA-per-particle layout on a full 8192-particle
window of the large-run workload.  Tolerance: 1e-4 relative over one window (FP32
rounding over Ns solves stopped at 1e-6).
"""
import dataclasses

import numpy as np
import pytest
import torch

from workloads import get_config, random_drift, random_increments, random_obs, random_state, u0_profile
from oracle import filter as OF
from tests.helpers import gpu_model, noise_poly_expected, oracle_model, rel_err, tdev

pytestmark = pytest.mark.gpu

F32_TOL = 1e-4


def _cfg(n, **over):
    return dataclasses.replace(get_config("cfg5_f32"), n=n, **over)


@pytest.mark.parametrize("n,layout,Ns,lam,mu", [(4096, "group", 10, True, 0.02), (4096, "group16", 4, True, 0.02),
                                                (2048, "group", 4, False, 0.02), (2048, "group16", 4, True, 0.02),
                                                (4096, "group", 3, True, 2.0), (1024, "group16", 10, True, 0.02),
                                                (1024, "group16", 3, True, 2.0)])
def test_group_window_matches_oracle(n, layout, Ns, lam, mu):
    cfg = _cfg(n, mu=mu)
    g = gpu_model(cfg, layout=layout)
    assert g.layout == layout and g.group_warps == n // (128 * g.group_cs)
    # both noise forms: the polynomials at n = 4096 (both layouts) and at n = 2048 with 16
    # nodes a lane, the tables elsewhere
    assert g.noise_form == ("poly" if noise_poly_expected(n, 2 * g.group_cs, cfg.K // 2) else "table")
    om = oracle_model(cfg)
    N = 3
    m0 = np.stack([om.m_from_u(u) for u in random_state(cfg, N, 31)])
    dW = random_increments(cfg, N, 32, steps=Ns)
    la = random_drift(cfg, N, 33, steps=Ns) if lam else None
    y = random_obs(cfg, 34)
    ref = om.ensemble_window(m0, dW, la)
    dt = g.dtype
    out = g.ensemble_step(tdev(m0, dt), tdev(dW, dt), None if la is None else tdev(la, dt), tdev(y, dt))
    torch.cuda.synchronize()
    assert rel_err(out["m"].cpu().numpy(), ref[0]) < F32_TOL
    assert rel_err(out["u"].cpu().numpy(), ref[1]) < F32_TOL
    assert np.all(out["status"].cpu().numpy() == 0)
    nll = OF.nll(ref[1], y, cfg.sigma)
    assert np.allclose(out["nll"].cpu().numpy(), nll, rtol=1e-3)
    if lam:
        assert np.allclose(out["logG"].cpu().numpy(), OF.girsanov_logG(la, dW, cfg.dt), rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("n,layout,K", [(2048, "group", 2), (4096, "group", 64), (4096, "group16", 6),
                                        (2048, "group16", 64), (1024, "group16", 8), (1024, "group16", 64),
                                        (4096, "group", 42)])
def test_group_noise_extremes_match_oracle(n, layout, K):
    # the lane-centred noise synthesis with one harmonic, an odd harmonic count and the largest
    # K (32 harmonics, the whole table), in both warp-group layouts; and the polynomial form at
    # the most harmonics it takes (21 at n = 4096: fit error 2^-30.3)
    cfg = _cfg(n, K=K)
    g = gpu_model(cfg, layout=layout)
    assert g.layout == layout
    assert g.noise_form == ("poly" if (n, K) == (4096, 42) else "table")
    assert (g.noise_form == "poly") == noise_poly_expected(n, 2 * g.group_cs, K // 2)
    om = oracle_model(cfg)
    N, Ns = 2, 3
    m0 = np.stack([om.m_from_u(u) for u in random_state(cfg, N, 41)])
    dW = random_increments(cfg, N, 42, steps=Ns)
    la = random_drift(cfg, N, 43, steps=Ns)
    ref = om.ensemble_window(m0, dW, la)
    dt = g.dtype
    out = g.ensemble_step(tdev(m0, dt), tdev(dW, dt), tdev(la, dt))
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    assert rel_err(out["m"].cpu().numpy(), ref[0]) < F32_TOL
    assert rel_err(out["u"].cpu().numpy(), ref[1]) < F32_TOL


def test_group_layouts_agree_with_cta_at_full_size():
    # the large-run window (n = 4096, N = 8192, K = 32, Ns = 10) in the warp-group layouts and
    # the one-CTA-per-particle layout: equal to FP32 rounding, the same Picard counts up to one
    # per step; three sampled particles recomputed by the oracle
    cfg = get_config("cfg5_f32")
    gg, g16, gc = gpu_model(cfg), gpu_model(cfg, layout="group16"), gpu_model(cfg, layout="cta")
    assert gg.layout == "group" and g16.layout == "group16" and gc.layout == "cta"
    N = cfg.N
    u0 = torch.tensor(u0_profile(cfg), dtype=torch.float32, device="cuda")
    m0, _ = gg.prior_sample(N, u0, 5, cfg.prior_scale)
    dW = gg.draw_increments(N, cfg.Ns, 9, 1, 0)
    y = gg.synth_obs(u0, 2, 1)
    c = gc.ensemble_step(m0, dW, None, y)
    scale_u, scale_m = c["u"].abs().max().item(), c["m"].abs().max().item()
    for g in (gg, g16):
        a = g.ensemble_step(m0, dW, None, y)
        torch.cuda.synchronize()
        assert (a["u"] - c["u"]).abs().max().item() < F32_TOL * scale_u
        assert (a["m"] - c["m"]).abs().max().item() < F32_TOL * scale_m
        assert torch.all(a["status"] == 0)
        assert (a["iters"] - c["iters"]).abs().max().item() <= cfg.Ns
        assert torch.allclose(a["nll"], c["nll"], rtol=1e-3)
    om = oracle_model(cfg)
    a = gg.ensemble_step(m0, dW, None, y)
    m0h, dWh, yh = m0.double().cpu().numpy(), dW.double().cpu().numpy(), y.double().cpu().numpy()
    for p in (0, 4099, N - 1):
        mref, uref, _, ok = om.window(m0h[p], dWh[p])
        assert ok
        assert rel_err(a["m"][p].cpu().numpy(), mref) < F32_TOL
        assert rel_err(a["u"][p].cpu().numpy(), uref) < F32_TOL
        nref = OF.nll(uref[None], yh, cfg.sigma)[0]
        assert abs(a["nll"][p].item() - nref) < 1e-3 * max(1.0, nref)


def test_group_nonfinite_and_nonconvergence_flags():
    cfg = _cfg(4096)
    g = gpu_model(cfg)
    om = oracle_model(cfg)
    m0 = np.stack([om.m_from_u(u) for u in random_state(cfg, 3, 41)])
    m0[1, 3000] = np.nan          # in the last warp of particle 1
    dW = random_increments(cfg, 3, 42, steps=2)
    out = g.ensemble_step(tdev(m0, g.dtype), tdev(dW, g.dtype))
    st = out["status"].cpu().numpy()
    assert st[1] & 2 and st[0] == 0 and st[2] == 0
    g1 = gpu_model(dataclasses.replace(cfg, max_iter=1))
    out = g1.ensemble_step(tdev(np.nan_to_num(m0), g.dtype), tdev(dW, g.dtype))
    assert np.all(out["status"].cpu().numpy() & 1)


def test_group_jitter_warm_start_matches_cold_start():
    # the jitter workspace: every proposal after the first starts its Picard iterations from the
    # previous proposal's converged per-step states (rho near one).  The proposals, and so the
    # decisions and the stored noise, are those of the cold start; the windows move only within
    # the Picard tolerance, with fewer iterations.  At rho < 0.99 the workspace is not used.
    cfg = _cfg(4096)
    g = gpu_model(cfg, layout="group")
    om = oracle_model(cfg)
    N = 64
    dt = g.dtype
    m0 = tdev(np.stack([om.m_from_u(u) for u in random_state(cfg, N, 61)]), dt)
    dW0 = tdev(random_increments(cfg, N, 62), dt)
    y = tdev(random_obs(cfg, 63), dt)

    def run(warm, rho):
        if warm:
            assert g.ensure_jitter_workspace(N, cfg.Ns)
        else:
            g.clear_jitter_workspace()
        d = dW0.clone()
        st = g.ensemble_step(m0, d, None, y)
        acc, it, status = g.jitter(m0, d, None, y, st["nll"], st["logG"], st["m"], st["u"], 0.5, rho, 5, 11, 100,
                                   want_iters=True)
        torch.cuda.synchronize()
        assert np.all(status.cpu().numpy() == 0)
        return acc.clone(), it.clone(), d, st

    cold, warm = run(False, 0.9999), run(True, 0.9999)
    assert torch.equal(cold[0], warm[0])
    assert 0 < int(cold[0].sum()) < 5 * N
    assert torch.equal(cold[2], warm[2])
    assert rel_err(warm[3]["u"].cpu().numpy(), cold[3]["u"].double().cpu().numpy()) < F32_TOL
    assert np.allclose(warm[3]["nll"].cpu().numpy(), cold[3]["nll"].cpu().numpy(), rtol=1e-4)
    assert int(warm[1].sum()) < 0.8 * int(cold[1].sum())
    cold2, warm2 = run(False, 0.5), run(True, 0.5)
    g.clear_jitter_workspace()
    for a, b in zip(cold2[:3], warm2[:3]):
        assert torch.equal(a, b)
    assert torch.equal(cold2[3]["u"], warm2[3]["u"]) and torch.equal(cold2[3]["nll"], warm2[3]["nll"])
