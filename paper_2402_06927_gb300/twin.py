"""Twin experiments: a truth trajectory, its observations, and filters that assimilate them.

``exp1`` runs Exp 1 of Sec. 4.1: the truth and the particles start from the initial
ensemble of Eq. init_solve (``SchModel.prior_exp1``), observations are taken every
window, and the bootstrap filter and the filter with adaptive tempering and PCN
jittering assimilate the same observations.  Every step the analysis ensemble is
compared with the truth by EMRE, RB and RES (Sec. 4.1.1).
"""
from __future__ import annotations

import time

import torch

from . import _lib
from .filter import EnsembleFilter


def truth_and_observations(g, Ns: int, T: int, seed: int):
    """The truth from member 0 of the Exp 1 ensemble under ``seed``, run T windows of Ns steps
    with Philox (seed, TAG_TRUTH) noise; observations of each window's end state with
    (seed, TAG_OBS) errors.  Returns (truths, ys), lists of T device vectors."""
    m_t, _ = g.prior_exp1(1, seed)
    truths, ys = [], []
    for c in range(T):
        out = g.ensemble_step(m_t, g.draw_increments(1, Ns, seed, _lib.TAG_TRUTH, c))
        m_t = out["m"]
        truths.append(out["u"][0].clone())
        ys.append(g.synth_obs(out["u"][0].contiguous(), seed, c))
    return truths, ys


def exp1(g, cfg, T: int, seed_truth: int = 2, seed_ens: int = 1, seed: int = 3):
    """Both filters of Exp 1 over T assimilation steps.  The bootstrap filter takes the whole
    step in one tempering stage (ESS threshold 1e-9), resamples and does not jitter; the other
    tempers to ESS >= cfg.ess_min with cfg.n_jitter PCN steps per stage.  Returns
    {name: dict(series [T, 3] EMRE/RB/RES on the host, stages [T], seconds)}."""
    truths, ys = truth_and_observations(g, cfg.Ns, T, seed_truth)
    m0, _ = g.prior_exp1(cfg.N, seed_ens)
    diag_ws = torch.empty(cfg.n, dtype=torch.float64, device="cuda")
    out = {}
    for name, ess_min, n_jitter in (("bootstrap", 1e-9, 0), ("tempering_jittering", cfg.ess_min, cfg.n_jitter)):
        f = EnsembleFilter(g, cfg.N, cfg.Ns, ess_min, cfg.rho, n_jitter, seed)
        f.set_state(m0)
        series = torch.empty((T, 3), dtype=torch.float64, device="cuda")
        stages = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c in range(T):
            st = f.cycle(ys[c], c)
            f.advance()
            series[c] = g.diagnostics(f.u_end, truths[c], ws=diag_ws)[:3]
            stages.append(len(st.stages))
        torch.cuda.synchronize()
        out[name] = dict(series=series.cpu().numpy(), stages=stages, seconds=time.perf_counter() - t0)
    out["initial"] = g.diagnostics(g.u_from_m(m0), truths[0], ws=diag_ws)[:3].cpu().numpy()
    return out
