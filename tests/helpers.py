"""Shared helpers for the GPU parity tests: build the library, make contexts."""
import numpy as np
import torch

from workloads import get_config, mode_amplitudes
from oracle.model import Model


def require_lib():
    from paper_2402_06927_gb300 import build
    build.build()
    from paper_2402_06927_gb300 import api
    return api


def gpu_model(cfg, **over):
    api = require_lib()
    return api.SchModel.from_config(cfg, **over)


def oracle_model(cfg, **over):
    kw = dict(tol=1e-13, max_iter=100)
    kw.update(noise_model=cfg.noise, kappa=cfg.kappa, eta=cfg.eta, matern_k=cfg.matern_k)
    kw.update(over)
    return Model(L=cfg.L, n=cfg.n, alpha=cfg.alpha, mu=cfg.mu, dt=cfg.dt, amps=mode_amplitudes(cfg), **kw)


def noise_poly_expected(n, H, K2, WNP=4):
    """Whether the warp-group kernels sum the mode noise of a lane with 2H nodes through
    polynomials (sch_noise_form), re-derived with numpy: per harmonic j, the Chebyshev
    interpolants in s = tau^2 of cos(x sqrt s) and sin(x sqrt s) / sqrt s (x = j d_max) must
    reproduce cos(j d) and sin(j d) at the lane's H offsets to 2^-30, and cost fewer packed
    FMAs than the tables."""
    Q = H // 2
    if K2 * WNP + Q * (2 * WNP - 1) >= K2 * 2 * Q:
        return False
    P = np.polynomial.polynomial
    dmax = 2 * np.pi * (H - 0.5) / n
    sn = 0.5 * (1 + np.cos(np.pi * (np.arange(WNP) + 0.5) / WNP))
    t = (np.arange(H) + 0.5) / (H - 0.5)
    err = 0.0
    for j in range(1, K2 + 1):
        x = j * dmax
        cc = P.polyfit(sn, np.cos(x * np.sqrt(sn)), WNP - 1)
        cs = P.polyfit(sn, np.sin(x * np.sqrt(sn)) / np.sqrt(sn), WNP - 1)
        err = max(err, np.abs(P.polyval(t * t, cc) - np.cos(x * t)).max(),
                  np.abs(t * P.polyval(t * t, cs) - np.sin(x * t)).max())
    return err <= 2.0 ** -30


def tdev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def nll_error_bound(nll, m_obs, u_scale, sigma, rel_tol):
    """Largest change of NLL = 1/2 sum_j ((u_j - y_j) / sigma)^2 when every observed u_j moves
    by at most rel_tol u_scale: by Cauchy-Schwarz, sum |r_j| |du_j| / sigma <= sqrt(2 NLL M)
    rel_tol u_scale / sigma (first order; the second-order term M (rel_tol u_scale / sigma)^2 / 2
    is added)."""
    d = rel_tol * u_scale / sigma
    return np.sqrt(2.0 * max(nll, 0.0) * m_obs) * d + 0.5 * m_obs * d * d


def pcn_generator(g):
    """The oracle generator that matches a GPU model's per-cell draws: Philox4x32-10 for the
    FP32 Matern noise, Philox4x64-10 otherwise."""
    import torch
    from oracle import rng as ORNG
    return ORNG.GEN32 if (g.noise == "matern" and g.dtype == torch.float32) else ORNG.GEN64


def jitter_moves_vs_oracle(g, om, cfg, m0d, dWd, lad, yd, theta, n_iter, seed, ctr, particles, field_tol, rho=None):
    """PCN jitter on the GPU one move at a time against the oracle, move by move.

    pf_jitter with n_iter = 1 and counter ctr + j is move j of one n_iter call (the
    proposal and the accept uniform of move j are keyed by ctr + j, and the state carries
    over), so the GPU state can be read between moves.  For every sampled particle p and
    move j the oracle replays the move from the GPU's current noise (its own window for the
    current state and for the proposal, Philox particle index p) and gives its decision and
    its Metropolis margin (w0 - w1) - log U.  Returns one record per (p, j):
    (p, j, gpu accepted, oracle accepted, margin, bound), where bound is the largest change
    of w0 - w1 that fields within field_tol (relative) can cause; and checks the new state of
    every move both sides accepted against the oracle's proposal window to field_tol."""
    import torch
    from oracle import filter as OF
    rho = cfg.rho if rho is None else rho
    gen = pcn_generator(g)
    st = g.ensemble_step(m0d, dWd, lad, yd)
    nll, logG, m_end, u_end = st["nll"], st["logG"], st["m"], st["u"]
    s0 = st["status"].cpu().numpy()
    assert np.all(s0 == 0), f"window status {np.unique(s0, return_counts=True)} at {np.nonzero(s0)[0][:8]}"
    m0h = m0d.double().cpu().numpy()
    yh = yd.double().cpu().numpy()
    lah = None if lad is None else lad.double().cpu().numpy()
    m_obs = int(np.sum(~np.isnan(yh)))
    out = []
    for j in range(n_iter):
        dW_before = dWd.double().cpu().numpy()
        acc, _, status = g.jitter(m0d, dWd, lad, yd, nll, logG, m_end, u_end, theta, rho, 1, seed, ctr + j)
        torch.cuda.synchronize()
        sj = status.cpu().numpy()
        assert np.all(sj == 0), f"move {j} status {np.unique(sj, return_counts=True)} at {np.nonzero(sj)[0][:8]}"
        acc = acc.cpu().numpy()
        for p in particles:
            la_p = None if lah is None else lah[p:p + 1]
            r = OF.jitter(om, m0h[p:p + 1], dW_before[p:p + 1], la_p, yh, cfg.sigma, theta, rho, 1, seed,
                          ctr + j, particle0=p, margins=True, gen=gen)
            dW_o, nll_o, _, _, u_o, acc_o, marg, prop_nll, prev_nll = r
            nll_cur = prev_nll[0, 0]
            u_scale = float(np.max(np.abs(u_o[0])))
            bound = theta * (nll_error_bound(nll_cur, m_obs, u_scale, cfg.sigma, field_tol)
                             + nll_error_bound(prop_nll[0, 0], m_obs, u_scale, cfg.sigma, field_tol))
            out.append((p, j, int(acc[p]), int(acc_o[0]), float(marg[0, 0]), float(bound)))
            if acc[p] == 1 and acc_o[0] == 1:
                assert rel_err(dWd[p].double().cpu().numpy(), dW_o[0]) < field_tol
                assert rel_err(u_end[p].double().cpu().numpy(), u_o[0]) < field_tol
                assert abs(nll[p].item() - nll_o[0]) <= nll_error_bound(nll_o[0], m_obs, u_scale, cfg.sigma,
                                                                        field_tol) + 1e-9 * max(1.0, nll_o[0])
    return out


def assert_decisions(records, exact):
    """Every move's decision equals the oracle's; with exact=False a move may differ only where
    the oracle's margin is within the bound the field tolerance allows."""
    bad = [r for r in records if r[2] != r[3] and (exact or abs(r[4]) > r[5])]
    assert not bad, f"decisions differ beyond the margin bound: {bad}"
