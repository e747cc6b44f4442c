"""Learned nudging proposal: training data, training, and the comparison with
optimiser nudging (host orchestration of library calls only).

* ``generate_pairs``: a twin experiment whose ensemble is advanced by the
  tempering + jittering filter; at every cycle pf_nudge (open-loop schedule)
  computes each particle's optimal drift for the cycle's observations, giving
  (u_start, y, lambda*) training pairs.
* ``train``: Adam on the network's kernels (nn_backward, nn_adam_step).
* ``run_nudged``: runs a twin experiment, nudging each cycle's ensemble with the
  trained network (nn_forward), with the network backed by the optimiser
  (pf_nudge instead whenever the network's forecast ESS falls below N/4), with
  the optimiser alone, or not at all, then tempering + jittering; reports
  cycles/s, the RMSE of the analysis mean against the truth, the ESS of the
  Girsanov-corrected weights before tempering and the fallback cycles.
"""
from __future__ import annotations

import time
from dataclasses import dataclass
from typing import Dict, List

import torch

from . import _lib
from .api import ProposalNet, SchModel
from .filter import EnsembleFilter


@dataclass
class Twin:
    """Truth trajectory and observations of a twin experiment (on the device)."""
    truths: List[torch.Tensor]
    ys: List[torch.Tensor]


def make_twin(g: SchModel, Ns: int, cycles: int, seed: int, u0: torch.Tensor) -> Twin:
    m_truth = g.m_from_u(u0[None].contiguous())
    truths, ys = [], []
    for c in range(cycles):
        dW = g.draw_increments(1, Ns, seed, _lib.TAG_TRUTH, c)
        out = g.ensemble_step(m_truth, dW)
        m_truth = out["m"]
        truths.append(out["u"][0].clone())
        ys.append(g.synth_obs(out["u"][0].contiguous(), seed, c))
    return Twin(truths, ys)


def generate_pairs(g: SchModel, N: int, Ns: int, cycles: int, seed: int, u0: torch.Tensor, ess_min: float,
                   rho: float, n_jitter: int, prior_scale: float, max_iter: int = 30, gtol: float = 1e-4,
                   keep: int = 0):
    """(U [P, n], Y [P, M], T [P, Ns, K]) with P = N cycles (or keep cycles: only every
    (N / keep)-th particle of each cycle's ensemble is nudged, which spreads the same number
    of pairs over more cycles, i.e. more observation vectors), plus generation statistics."""
    twin = make_twin(g, Ns, cycles, seed, u0)
    f = EnsembleFilter(g, N, Ns, ess_min, rho, n_jitter, seed)
    m0, _ = g.prior_sample(N, u0, seed, prior_scale)
    f.set_state(m0)
    U, Y, T = [], [], []
    t0 = time.perf_counter()
    iters = []
    stride = N // keep if 0 < keep < N else 1
    for c in range(cycles):
        y = twin.ys[c]
        m_sel = f.m_start[::stride].contiguous()
        u_start = g.u_from_m(m_sel)
        nd = g.nudge(m_sel, y, Ns, mode="open_loop", max_iter=max_iter, gtol=gtol, seed=seed,
                     ctr=1_000_000 + c)
        U.append(u_start.float())
        Y.append(y.float()[None].expand(m_sel.shape[0], -1).contiguous())
        T.append(nd["lam"].float())
        iters.append(nd["iters"].float().mean().item())
        f.set_drift(None)
        f.cycle(y, c)
        f.advance()
    torch.cuda.synchronize()
    stats = dict(seconds=time.perf_counter() - t0, mean_lbfgs_iters=sum(iters) / len(iters))
    return torch.cat(U), torch.cat(Y), torch.cat(T), stats


def train(net: ProposalNet, U, Y, T, epochs: int = 20, batch: int = 256, lr: float = 1e-3, seed: int = 0,
          val_frac: float = 0.1) -> Dict[str, float]:
    P = U.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(P, generator=g).cuda()
    nval = max(batch, int(val_frac * P))
    val, tr = perm[:nval], perm[nval:]
    t0 = time.perf_counter()
    last = None
    for ep in range(epochs):
        order = tr[torch.randperm(tr.numel(), generator=g).cuda()]
        rate = lr * (0.5 ** (ep // max(1, epochs // 3)))
        for i in range(0, order.numel() - batch + 1, batch):
            idx = order[i:i + batch]
            last = net.train_step(U[idx].contiguous(), Y[idx].contiguous(), T[idx].contiguous(), lr=rate)
    torch.cuda.synchronize()
    vl = []
    for i in range(0, val.numel() - batch + 1, batch):
        idx = val[i:i + batch]
        loss, _ = net.loss_and_grad(U[idx].contiguous(), Y[idx].contiguous(), T[idx].contiguous())
        vl.append(loss.item())
    tvar = 0.5 * T[val].float().pow(2).sum(dim=(1, 2)).mean().item()
    return dict(seconds=time.perf_counter() - t0, train_loss=float(last.item()) if last is not None else None,
                val_loss=sum(vl) / max(1, len(vl)), val_target_energy=tvar)


def run_nudged(g: SchModel, source: str, net: ProposalNet, N: int, Ns: int, cycles: int, seed: int,
               u0: torch.Tensor, ess_min: float, rho: float, n_jitter: int, prior_scale: float,
               twin: Twin, max_iter: int = 30, gtol: float = 1e-4, refine: int = 1,
               fallback_frac: float = 0.25):
    """Cycles of a nudged tempering + jittering filter.

    source: 'learned' (network drift), 'learned_fb' (network drift, and the optimiser
    instead for a cycle whose forecast ESS under the network's drift falls below
    fallback_frac N), 'optimiser' (pf_nudge from zero), 'hybrid' (pf_nudge started
    from the network's drift, `refine` L-BFGS iterations) or 'none'.
    """
    f = EnsembleFilter(g, N, Ns, ess_min, rho, n_jitter, seed)
    m0, _ = g.prior_sample(N, u0, seed, prior_scale)
    f.set_state(m0)
    diag_ws = torch.empty(g.n, dtype=torch.float64, device="cuda")
    diag = torch.empty(8, dtype=torch.float64, device="cuda")
    rmse, ess0, stages = [], [], []
    fallbacks = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in range(cycles):
        y = twin.ys[c]
        dW = None
        done = False
        if source in ("learned", "learned_fb"):
            u_start = g.u_from_m(f.m_start)
            lam = net.forward(u_start, y)
            f.set_drift(lam.to(g.dtype))
            dW = g.draw_increments(N, Ns, seed, _lib.TAG_NUDGE, 1_000_000 + c)
            if source == "learned_fb":
                # the forecast under the network's drift; if its Girsanov-corrected weights
                # have ESS below fallback_frac N, the optimiser nudges this cycle instead
                f.forecast(y, dW)
                done = True
                if f.forecast_ess() < fallback_frac * N:
                    nd = g.nudge(f.m_start, y, Ns, mode="open_loop", max_iter=max_iter, gtol=gtol, seed=seed,
                                 ctr=1_000_000 + c)
                    f.set_drift(nd["lam"])
                    dW = nd["dW"]
                    done = False
                    fallbacks += 1
        elif source in ("optimiser", "hybrid"):
            lam0 = None
            if source == "hybrid":
                lam0 = net.forward(g.u_from_m(f.m_start), y).to(g.dtype)
            nd = g.nudge(f.m_start, y, Ns, mode="open_loop", max_iter=max_iter if source == "optimiser" else refine,
                         gtol=gtol, seed=seed, ctr=1_000_000 + c, lam0=lam0)
            f.set_drift(nd["lam"])
            dW = nd["dW"]
        else:
            f.set_drift(None)
        st = f.cycle(y, c, dW=dW, forecast_done=done)
        ess0.append(st.ess0)
        stages.append(len(st.stages))
        f.advance()
        g.diagnostics(f.u_end, twin.truths[c], ws=diag_ws, out=diag)
        rmse.append(diag[3])
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    return dict(cycles_per_s=cycles / secs, rmse=float(torch.stack(rmse).mean().item()),
                mean_stages=sum(stages) / len(stages), mean_forecast_ess=sum(ess0) / len(ess0),
                fallback_cycles=fallbacks)
