"""Host driver of one assimilation cycle on the GPU (Sec. 3.1 of the paper).

The cycle works on the (X_start, dW) representation of a particle
(Sec. 3.1.2): draw the window noise, propagate every particle through the
window (with the fused likelihood epilogue), then repeat adaptive tempering,
systematic resampling and PCN jittering until the temperature reaches one;
finally the end state becomes the next window's start.  Every step is a call
into the CUDA library.  By default the first `eager_stages` stages are all
enqueued at once as device-gated stages (a stage that starts at temperature one
does nothing), and the host reads the stages' tempering results back once per
cycle; only a cycle that needs more stages continues stage by stage, reading back
each stage's 40-byte result to decide whether another is needed.
"""
from __future__ import annotations

import ctypes as ct
from dataclasses import dataclass, field
from typing import List, Optional

import torch

from . import _lib
from .api import SchModel, pf_gather_rows, pf_resample, pf_resample_gated, pf_temper, pf_temper_dev


@dataclass
class StageStats:
    dtheta: float
    ess: float
    theta: float


@dataclass
class CycleStats:
    stages: List[StageStats] = field(default_factory=list)
    forward_steps: int = 0      # particle-timesteps propagated in the cycle (incl. PCN re-runs)
    launches: int = 0           # library kernels launched by the cycle
    accepts: Optional[torch.Tensor] = None
    ess0: Optional[float] = None  # ESS of the untempered (Girsanov-corrected) forecast weights


class KernelTimer:
    """CUDA events around the jitter launches of a cycle (on the launching stream);
    launches of inactive device-gated stages are dropped after the cycle."""

    def __init__(self):
        self.pairs = []
        self.iters = []

    def elapsed_ms(self):
        return [a.elapsed_time(b) for a, b in self.pairs]


class EnsembleFilter:
    """GPU state of an N-particle tempering + jittering filter."""

    def __init__(self, model: SchModel, N: int, Ns: int, ess_min: float, rho: float, n_jitter: int,
                 seed: int, lam: Optional[torch.Tensor] = None, temper_mode: str = "largest",
                 eager_stages: int = 2, warm_jitter: bool = True):
        self.model, self.N, self.Ns = model, N, Ns
        # warm_jitter: the model's jitter calls start each proposal after the first from the
        # previous proposal's per-step states, where the layout supports it (a workspace the
        # model keeps; the warp-group layout only)
        self.warm_jitter = bool(warm_jitter) and model.ensure_jitter_workspace(N, Ns)
        self.temper_mode = temper_mode   # "largest" or "halving" (pf_temper / pf_temper_halving)
        self.eager_stages = eager_stages  # device-gated stages enqueued at once (0: stage by stage)
        self.ess_min, self.rho, self.n_jitter, self.seed = ess_min, rho, n_jitter, seed
        dt, dev, n, K = model.dtype, torch.device("cuda"), model.n, model.K

        def fld():
            return torch.zeros((N, n), dtype=dt, device=dev)

        self.m_start, self.m_end, self.u_end = fld(), fld(), fld()
        self.dW = torch.zeros((N, Ns, K), dtype=dt, device=dev)
        self.lam = lam
        self.nll = torch.zeros(N, dtype=torch.float64, device=dev)
        self.logG = torch.zeros(N, dtype=torch.float64, device=dev)
        # second copies for out-of-place resampling gathers
        self._b = dict(m_start=fld(), m_end=fld(), u_end=fld(),
                       dW=torch.zeros_like(self.dW), nll=torch.zeros_like(self.nll),
                       logG=torch.zeros_like(self.logG))
        if lam is not None:
            self._b["lam"] = torch.zeros_like(lam)
        self.wbar = torch.zeros(N, dtype=torch.float64, device=dev)
        self.tout = torch.zeros(4, dtype=torch.float64, device=dev)
        self.tout_host = torch.zeros(4, dtype=torch.float64).pin_memory()
        S = max(1, eager_stages)   # mean stages per cycle at the bench size: 1.24
        self.touts = torch.zeros((S, 5), dtype=torch.float64, device=dev)
        self.touts_host = torch.zeros((S, 5), dtype=torch.float64).pin_memory()
        self.theta0 = torch.zeros(1, dtype=torch.float64, device=dev)
        # recorded after the last launch of each cycle: the end of the cycle's device work
        self.end_event = torch.cuda.Event(enable_timing=True)
        self.idx = torch.zeros(N, dtype=torch.int32, device=dev)
        self.accepts = torch.zeros(N, dtype=torch.int32, device=dev)
        self.status = torch.zeros(N, dtype=torch.int32, device=dev)

    def set_state(self, m_start: torch.Tensor) -> None:
        self.m_start.copy_(m_start)

    def set_drift(self, lam: Optional[torch.Tensor]) -> None:
        """Nudging drift of the coming window (None: no nudging)."""
        if lam is None:
            self.lam = None
            self._b.pop("lam", None)
            return
        if self.lam is None or self.lam.shape != lam.shape:
            self.lam = torch.empty_like(lam)
            self._b["lam"] = torch.empty_like(lam)
        self.lam.copy_(lam)

    def _gather_all(self) -> None:
        names = ["m_start", "m_end", "u_end", "dW", "nll", "logG"] + (["lam"] if self.lam is not None else [])
        for name in names:
            cur = getattr(self, name)
            nxt = self._b[name]
            pf_gather_rows(self.idx, cur, nxt)
            setattr(self, name, nxt)
            self._b[name] = cur

    def _jitter(self, y, theta, stage_ctr, timer, tstate=None):
        m = self.model
        iters = None
        if timer is not None:
            iters = torch.zeros(self.N, dtype=torch.int32, device=self.nll.device)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record()
        m.jitter(self.m_start, self.dW, self.lam, y, self.nll, self.logG, self.m_end, self.u_end, theta,
                 self.rho, self.n_jitter, self.seed, stage_ctr * self.n_jitter, accepts=self.accepts,
                 status=self.status, iters=iters, tstate=tstate)
        if timer is not None:
            ev1.record()
            timer.pairs.append((ev0, ev1))
            timer.iters.append(iters)

    def _resample(self, stage_ctr: int) -> None:
        pf_resample(self.wbar, self.seed, stage_ctr, idx=self.idx)
        self._gather_all()

    def forecast(self, y: torch.Tensor, dW: torch.Tensor) -> None:
        """The window's forecast into the filter's own buffers: dW copied in, then every
        particle propagated from m_start with the current drift (sch_ensemble_step with the
        fused likelihood); a following ``cycle(..., forecast_done=True)`` starts from it."""
        self.dW.copy_(dW)
        self.model.ensemble_step(self.m_start, self.dW, self.lam, y, m_out=self.m_end, u_out=self.u_end,
                                 nll=self.nll, logG=self.logG, status=self.status, want_iters=False)

    def forecast_ess(self) -> float:
        """ESS of the Girsanov-corrected weights exp(-(nll - logG)) of the current forecast
        (pf_temper at theta = 0: its out[3]); reads 8 bytes back to the host."""
        pf_temper(self.nll, self.logG, 0.0, self.ess_min, wbar=self.wbar, out=self.tout, mode=self.temper_mode)
        self.tout_host.copy_(self.tout, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        return float(self.tout_host[3])

    def cycle(self, y: torch.Tensor, cycle: int, max_stages: int = 64,
              timer: Optional[KernelTimer] = None, dW: Optional[torch.Tensor] = None,
              post=None, forecast_done: bool = False) -> CycleStats:
        """One assimilation cycle.  ``dW`` (optional) supplies the window increments
        (e.g. the ones revealed by pf_nudge); otherwise they are drawn from the prior.
        With ``forecast_done`` the filter's buffers already hold this window's forecast
        (``forecast``) and it is not run again.
        ``post`` (optional, no arguments) enqueues work on the analysis ensemble, such as
        diagnostics and their copy to the host, on the current stream.  It is called right
        after the device-gated stages are enqueued, before the cycle waits for them, and
        again after any later stage, so the work it enqueued last sees the final analysis."""
        m = self.model
        st = CycleStats()
        if not (y.is_cuda and y.dtype == m.dtype and y.numel() == m.M and y.is_contiguous()):
            raise ValueError(f"y must be a contiguous CUDA {m.dtype} vector of {m.M} observations")
        # the forecast through the C ABI directly: the filter's own buffers have the shapes and
        # types the library expects, so the argument checks of SchModel are not repeated (they
        # cost about 20 us of host time per call, while the GPU waits for the cycle's first work)
        L = _lib.lib()
        stream = torch.cuda.current_stream().cuda_stream
        if not forecast_done:
            if dW is None:
                _lib.check(L.sch_draw_increments(m.handle, self.N, self.Ns, self.seed, _lib.TAG_PRIOR_DW, cycle, 0,
                                                 self.dW.data_ptr(), stream), "sch_draw_increments")
            else:
                self.dW.copy_(dW)
            _lib.check(L.sch_ensemble_step(m.handle, self.N, self.Ns, self.m_start.data_ptr(),
                                           self.m_end.data_ptr(), self.u_end.data_ptr(), self.dW.data_ptr(),
                                           None if self.lam is None else self.lam.data_ptr(), y.data_ptr(),
                                           self.nll.data_ptr(), self.logG.data_ptr(), None, self.status.data_ptr(),
                                           stream), "sch_ensemble_step")
            st.launches += 2
        st.forward_steps += self.N * self.Ns
        st.ess0 = None
        theta, k = 0.0, 0
        if self.eager_stages > 0:
            # device-gated stages enqueued by one library call (pf_gated_stages): stage k
            # reads its temperature from stage k-1's result and does nothing but copy the
            # rows once the temperature is one; the host reads all results back once
            S = min(self.eager_stages, max_stages)
            names = ["m_start", "m_end", "u_end", "dW", "nll", "logG", "lam"]
            cur = [getattr(self, nm) if nm != "lam" else self.lam for nm in names]
            nxt = [self._b.get(nm) for nm in names]
            ptr = lambda t: None if t is None else t.data_ptr()
            bufs_a = (ct.c_void_p * 7)(*[ptr(t) for t in cur])
            bufs_b = (ct.c_void_p * 7)(*[ptr(t) for t in nxt])
            iters = evs = None
            if timer is not None:
                iters = torch.zeros((S, self.N), dtype=torch.int32, device=self.nll.device)
                pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                         for _ in range(S)]
                for a, b in pairs:   # create the events; the library records them again
                    a.record()
                    b.record()
                evs = (ct.c_void_p * (2 * S))(*[e.cuda_event for ab in pairs for e in ab])
            _lib.check(_lib.lib().pf_gated_stages(
                m.handle, self.N, self.Ns, S, 0, self.ess_min, {"largest": 0, "halving": 1}[self.temper_mode],
                self.rho, self.n_jitter, self.seed, cycle, ct.c_void_p(y.data_ptr()), bufs_a, bufs_b,
                ct.c_void_p(self.theta0.data_ptr()), ct.c_void_p(self.wbar.data_ptr()),
                ct.c_void_p(self.idx.data_ptr()), ct.c_void_p(self.touts.data_ptr()),
                ct.c_void_p(self.accepts.data_ptr()), ct.c_void_p(ptr(iters)), ct.c_void_p(self.status.data_ptr()),
                evs, ct.c_void_p(torch.cuda.current_stream().cuda_stream)), "pf_gated_stages")
            self.end_event.record()
            if S % 2 == 1:   # every stage gathers a -> b: an odd count leaves the state in the b copies
                for nm, c, n2 in zip(names, cur, nxt):
                    if c is None:
                        continue
                    setattr(self, nm, n2)
                    self._b[nm] = c
            st.launches += S * 4
            if post is not None:
                post()
            n0 = len(timer.pairs) if timer is not None else 0
            if timer is not None:
                timer.pairs.extend(pairs)
                timer.iters.extend(iters[k] for k in range(S))
            self.touts_host.copy_(self.touts, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            touts = self.touts_host.tolist()
            for k in range(S):
                d, e, theta_new, e_rest, active = touts[k]
                if active == 0.0:
                    if timer is not None:
                        del timer.pairs[n0 + k:], timer.iters[n0 + k:]
                    break
                st.forward_steps += self.N * self.Ns * self.n_jitter
                st.stages.append(StageStats(d, e, theta_new))
                if k == 0:
                    st.ess0 = e_rest
                theta = theta_new
            k = len(st.stages)
        while theta < 1.0 and k < max_stages:
            pf_temper(self.nll, self.logG, theta, self.ess_min, wbar=self.wbar, out=self.tout, mode=self.temper_mode)
            self.tout_host.copy_(self.tout, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            d, e, theta_new = self.tout_host[:3].tolist()
            stage_ctr = cycle * 1024 + k
            self._resample(stage_ctr)
            theta = theta_new
            self._jitter(y, theta, stage_ctr, timer)
            self.end_event.record()
            st.forward_steps += self.N * self.Ns * self.n_jitter
            st.launches += 2 + len(self._b) + 1
            st.stages.append(StageStats(d, e, theta))
            if k == 0:
                st.ess0 = float(self.tout_host[3])
            k += 1
        if post is not None and (self.eager_stages == 0 or len(st.stages) > min(self.eager_stages, max_stages)):
            # stages after the gated ones (or no gated ones): the work runs on the final analysis
            post()
            torch.cuda.current_stream().synchronize()
        st.accepts = self.accepts
        return st

    def advance(self) -> None:
        """The end of this window becomes the start of the next (X_start <- X_end)."""
        self.m_start, self.m_end = self.m_end, self.m_start
