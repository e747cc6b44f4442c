"""Twin experiments: a truth trajectory, its observations, and filters that assimilate them.

``exp1`` runs Exp 1 of Sec. 4.1: the truth and the particles start from the initial
ensemble of Eq. init_solve (``SchModel.prior_exp1``), observations are taken every
window, and the bootstrap filter and the filter with adaptive tempering and PCN
jittering assimilate the same observations.  Every step the analysis ensemble is
compared with the truth by EMRE, RB and RES (Sec. 4.1.1).  ``exp2`` is the same with
Exp 2's half-domain observations: only the points in [0, L/2] are observed (the
others NaN), and the ensemble mean's error is also split between the two halves.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import _lib
from .filter import EnsembleFilter


def truth_and_observations(g, Ns: int, T: int, seed: int, upto=None):
    """The truth from member 0 of the Exp 1 ensemble under ``seed``, run T windows of Ns steps
    with Philox (seed, TAG_TRUTH) noise; observations of each window's end state with
    (seed, TAG_OBS) errors, the points x_j > upto L not observed (NaN) when upto is given.
    Returns (truths, ys), lists of T device vectors."""
    m_t, _ = g.prior_exp1(1, seed)
    truths, ys = [], []
    for c in range(T):
        out = g.ensemble_step(m_t, g.draw_increments(1, Ns, seed, _lib.TAG_TRUTH, c))
        m_t = out["m"]
        truths.append(out["u"][0].clone())
        y = g.synth_obs(out["u"][0].contiguous(), seed, c)
        if upto is not None:
            y[int(upto * g.M) + 1:] = float("nan")
        ys.append(y)
    return truths, ys


def exp1(g, cfg, T: int, seed_truth: int = 2, seed_ens: int = 1, seed: int = 3, upto=None):
    """Both filters of Exp 1 over T assimilation steps.  The bootstrap filter takes the whole
    step in one tempering stage (ESS threshold 1e-9), resamples and does not jitter; the other
    tempers to ESS >= cfg.ess_min with cfg.n_jitter PCN steps per stage.  Returns
    {name: dict(series [T, 3] EMRE/RB/RES, halves [T, 2] relative error of the ensemble mean
    on [0, L/2] and (L/2, L), stages [T], seconds)}, host arrays."""
    truths, ys = truth_and_observations(g, cfg.Ns, T, seed_truth, upto)
    m0, _ = g.prior_exp1(cfg.N, seed_ens)
    diag_ws = torch.empty(cfg.n, dtype=torch.float64, device="cuda")
    half = cfg.n // 2 + 1
    out = {}
    for name, ess_min, n_jitter in (("bootstrap", 1e-9, 0), ("tempering_jittering", cfg.ess_min, cfg.n_jitter)):
        f = EnsembleFilter(g, cfg.N, cfg.Ns, ess_min, cfg.rho, n_jitter, seed)
        f.set_state(m0)
        series = torch.empty((T, 3), dtype=torch.float64, device="cuda")
        means = torch.empty((T, cfg.n), dtype=torch.float64, device="cuda")
        stages = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for c in range(T):
            st = f.cycle(ys[c], c)
            f.advance()
            series[c] = g.diagnostics(f.u_end, truths[c], ws=diag_ws)[:3]
            means[c] = diag_ws      # the diagnostics leave the ensemble mean in their workspace
            stages.append(len(st.stages))
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        tr = torch.stack(truths).double().cpu().numpy()
        mn = means.cpu().numpy()
        halves = np.stack([np.linalg.norm(mn[:, :half] - tr[:, :half], axis=1) / np.linalg.norm(tr[:, :half], axis=1),
                           np.linalg.norm(mn[:, half:] - tr[:, half:], axis=1) / np.linalg.norm(tr[:, half:], axis=1)],
                          axis=1)
        out[name] = dict(series=series.cpu().numpy(), halves=halves, stages=stages, seconds=el)
    out["initial"] = g.diagnostics(g.u_from_m(m0), truths[0], ws=diag_ws)[:3].cpu().numpy()
    return out


def exp2(g, cfg, T: int, **kw):
    """Exp 2 of Sec. 4.1: ``exp1`` with only [0, L/2] observed."""
    return exp1(g, cfg, T, upto=0.5, **kw)
