"""Python binding of the C ABI (include/sch.h): argument marshalling only.

Every function takes CUDA tensors, checks shapes and dtypes, passes raw device
pointers and the current CUDA stream to the library, and raises on a
non-zero status.  No arithmetic of the method happens here.
"""
from __future__ import annotations

import ctypes as ct
from typing import Optional, Sequence

import torch

from . import _lib
from ._lib import NNShape, SCH_F32, SCH_F64, SchParams, check, lib


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ct.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ct.c_void_p(s.cuda_stream)


def _need(t: torch.Tensor, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class SchModel:
    """A library context for one set of model and observation parameters."""

    def __init__(self, L: float, n: int, alpha: float, mu: float, dt: float, amps: Sequence[float],
                 M: int, sigma: float, tol: float, max_iter: int, dtype: str = "f32", solver: str = "auto",
                 layout: str = "auto", noise: str = "modes", kappa: float = 1.0, eta: float = 1.0,
                 matern_k: int = 3):
        p = SchParams()
        p.L, p.n, p.alpha, p.mu, p.dt = L, n, alpha, mu, dt
        p.K = 2 * len(amps)
        for j, a in enumerate(amps):
            p.amps[j] = float(a)
        p.M, p.sigma, p.tol, p.max_iter = M, sigma, tol, max_iter
        p.dtype = SCH_F32 if dtype == "f32" else SCH_F64
        p.solver = {"auto": 0, "li": 1, "ea": 2}[solver]
        p.layout = {"auto": 0, "cta": 1, "warp": 2, "group": 3, "group16": 4}[layout]
        p.noise = {"modes": 0, "matern": 1}[noise]
        p.kappa, p.eta, p.matern_k = kappa, eta, matern_k
        self.params = p
        self.n, self.M, self.dt = n, M, dt
        self.dtype = torch.float32 if dtype == "f32" else torch.float64
        h = ct.c_void_p()
        check(lib().sch_create(ct.byref(p), ct.byref(h)), "sch_create")
        self._h = h
        # the kernel layout the library chose: "warp" (one warp per particle), "group" or
        # "group16" (n / 1024 or n / 512 warps per particle) or "cta"
        self.layout = {1: "cta", 2: "warp", 3: "group", 4: "group16"}[lib().sch_layout(h)]
        self.group_cs = 8 if self.layout == "group" else 4
        self.group_warps = n // (128 * self.group_cs) if self.layout.startswith("group") else 0
        # Brownian motions per step, the last axis of every dW and lambda: K mode
        # functions, or one per cell for the Matern noise
        self.K = int(lib().sch_noise_dim(h))
        self.noise = noise
        # how the warp and warp-group kernels sum the mode noise at a lane's nodes:
        # "table" (tabulated cos/sin of the node offsets), "poly" (host-fitted polynomials
        # of the offsets) or "other" (the CTA layout, the Matern noise)
        self.noise_form = {0: "other", 1: "table", 2: "poly"}[lib().sch_noise_form(h)]

    @classmethod
    def from_config(cls, cfg, **over):
        from workloads import mode_amplitudes
        kw = dict(L=cfg.L, n=cfg.n, alpha=cfg.alpha, mu=cfg.mu, dt=cfg.dt, amps=list(mode_amplitudes(cfg)),
                  M=cfg.M, sigma=cfg.sigma, tol=cfg.tol, max_iter=cfg.max_iter, dtype=cfg.dtype,
                  noise=cfg.noise, kappa=cfg.kappa, eta=cfg.eta, matern_k=cfg.matern_k)
        kw.update(over)
        return cls(**kw)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().sch_destroy(self._h)
            self._h = ct.c_void_p()
        self._jws = None

    def jitter_workspace_bytes(self, N: int, nsteps: int) -> int:
        """Bytes of the optional jitter workspace for N particles and nsteps steps (0 where the
        layout does not use one)."""
        return int(lib().sch_jitter_workspace_bytes(self._h, N, nsteps))

    def ensure_jitter_workspace(self, N: int, nsteps: int) -> bool:
        """Give the context a jitter workspace for up to N particles and nsteps steps (device
        memory kept by this object): later jitter calls warm-start their proposals' Picard
        iterations from the previous proposal of the call.  Returns whether the layout uses it."""
        need = self.jitter_workspace_bytes(N, nsteps)
        if need == 0:
            return False
        cur = getattr(self, "_jws", None)
        if cur is None or cur.numel() < need:
            self._jws = torch.empty(need, dtype=torch.uint8, device="cuda")
            check(lib().sch_set_jitter_workspace(self._h, _ptr(self._jws), need), "sch_set_jitter_workspace")
        return True

    def clear_jitter_workspace(self) -> None:
        """Every jitter proposal starts from the steps' start states again."""
        check(lib().sch_set_jitter_workspace(self._h, None, 0), "sch_set_jitter_workspace")
        self._jws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ #
    def u_from_m(self, m: torch.Tensor, u: Optional[torch.Tensor] = None) -> torch.Tensor:
        N = m.shape[0]
        _need(m, self.dtype, (N, self.n), "m")
        u = torch.empty_like(m) if u is None else u
        check(lib().sch_u_from_m(self._h, N, _ptr(m), _ptr(u), _stream()), "sch_u_from_m")
        return u

    def m_from_u(self, u: torch.Tensor, m: Optional[torch.Tensor] = None) -> torch.Tensor:
        N = u.shape[0]
        _need(u, self.dtype, (N, self.n), "u")
        m = torch.empty_like(u) if m is None else m
        check(lib().sch_m_from_u(self._h, N, _ptr(u), _ptr(m), _stream()), "sch_m_from_u")
        return m

    def draw_increments(self, N: int, nsteps: int, seed: int, tag: int, ctr: int, particle0: int = 0,
                        out: Optional[torch.Tensor] = None) -> torch.Tensor:
        out = torch.empty((N, nsteps, self.K), dtype=self.dtype, device="cuda") if out is None else out
        _need(out, self.dtype, (N, nsteps, self.K), "dW")
        check(lib().sch_draw_increments(self._h, N, nsteps, seed, tag, ctr, particle0, _ptr(out), _stream()),
              "sch_draw_increments")
        return out

    def ensemble_step(self, m: torch.Tensor, dW: torch.Tensor, lam: Optional[torch.Tensor] = None,
                      y: Optional[torch.Tensor] = None, m_out: Optional[torch.Tensor] = None,
                      u_out: Optional[torch.Tensor] = None, nll: Optional[torch.Tensor] = None,
                      logG: Optional[torch.Tensor] = None, iters: Optional[torch.Tensor] = None,
                      status: Optional[torch.Tensor] = None, want_iters: bool = True):
        """sch_ensemble_step: returns dict(m, u, nll, logG, iters, status)."""
        N = m.shape[0]
        nsteps = dW.shape[1]
        _need(m, self.dtype, (N, self.n), "m")
        _need(dW, self.dtype, (N, nsteps, self.K), "dW")
        if lam is not None:
            _need(lam, self.dtype, (N, nsteps, self.K), "lambda")
        m_out = torch.empty_like(m) if m_out is None else m_out
        u_out = torch.empty_like(m) if u_out is None else u_out
        _need(m_out, self.dtype, (N, self.n), "m_out")
        _need(u_out, self.dtype, (N, self.n), "u_out")
        if y is not None:
            _need(y, self.dtype, (self.M,), "y")
            nll = torch.empty(N, dtype=torch.float64, device=m.device) if nll is None else nll
            logG = torch.empty(N, dtype=torch.float64, device=m.device) if logG is None else logG
            _need(nll, torch.float64, (N,), "nll")
            _need(logG, torch.float64, (N,), "logG")
        else:
            nll = logG = None
        if iters is None and want_iters:
            iters = torch.empty(N, dtype=torch.int32, device=m.device)
        status = torch.empty(N, dtype=torch.int32, device=m.device) if status is None else status
        check(lib().sch_ensemble_step(self._h, N, nsteps, _ptr(m), _ptr(m_out), _ptr(u_out), _ptr(dW), _ptr(lam),
                                      _ptr(y), _ptr(nll), _ptr(logG), _ptr(iters), _ptr(status), _stream()),
              "sch_ensemble_step")
        return dict(m=m_out, u=u_out, nll=nll, logG=logG, iters=iters, status=status)

    def loglik(self, u: torch.Tensor, y: torch.Tensor, dW: Optional[torch.Tensor] = None,
               lam: Optional[torch.Tensor] = None):
        N = u.shape[0]
        _need(u, self.dtype, (N, self.n), "u")
        _need(y, self.dtype, (self.M,), "y")
        nsteps = 0 if dW is None else dW.shape[1]
        nll = torch.empty(N, dtype=torch.float64, device=u.device)
        logG = torch.empty(N, dtype=torch.float64, device=u.device)
        check(lib().sch_loglik(self._h, N, _ptr(u), _ptr(y), _ptr(dW), _ptr(lam), nsteps, _ptr(nll), _ptr(logG),
                               _stream()), "sch_loglik")
        return nll, logG

    def jitter(self, m_start, dW, lam, y, nll, logG, m_end, u_end, theta: float, rho: float, n_iter: int,
               seed: int, ctr: int, want_iters: bool = False, accepts=None, iters=None, status=None,
               tstate: Optional[torch.Tensor] = None):
        """pf_jitter: updates dW, nll, logG, m_end, u_end in place; returns (accepts, iters, status)."""
        N, nsteps, K = dW.shape
        _need(m_start, self.dtype, (N, self.n), "m_start")
        _need(dW, self.dtype, (N, nsteps, self.K), "dW")
        _need(m_end, self.dtype, (N, self.n), "m_end")
        _need(u_end, self.dtype, (N, self.n), "u_end")
        _need(y, self.dtype, (self.M,), "y")
        _need(nll, torch.float64, (N,), "nll")
        _need(logG, torch.float64, (N,), "logG")
        if lam is not None:
            _need(lam, self.dtype, (N, nsteps, self.K), "lambda")
        acc = torch.empty(N, dtype=torch.int32, device=dW.device) if accepts is None else accepts
        if iters is None and want_iters:
            iters = torch.empty(N, dtype=torch.int32, device=dW.device)
        status = torch.empty(N, dtype=torch.int32, device=dW.device) if status is None else status
        if tstate is not None:
            # device-gated stage: theta = tstate[2], nothing done when tstate[4] == 0
            check(lib().pf_jitter_dev(self._h, N, nsteps, n_iter, _ptr(tstate), rho, seed, ctr, _ptr(m_start),
                                      _ptr(dW), _ptr(lam), _ptr(y), _ptr(nll), _ptr(logG), _ptr(m_end),
                                      _ptr(u_end), _ptr(acc), _ptr(iters), _ptr(status), _stream()),
                  "pf_jitter_dev")
        else:
            check(lib().pf_jitter(self._h, N, nsteps, n_iter, theta, rho, seed, ctr, _ptr(m_start), _ptr(dW),
                                  _ptr(lam), _ptr(y), _ptr(nll), _ptr(logG), _ptr(m_end), _ptr(u_end), _ptr(acc),
                                  _ptr(iters), _ptr(status), _stream()), "pf_jitter")
        return acc, iters, status

    def synth_obs(self, u: torch.Tensor, seed: int, ctr: int, y: Optional[torch.Tensor] = None):
        _need(u, self.dtype, (self.n,), "u")
        y = torch.empty(self.M, dtype=self.dtype, device=u.device) if y is None else y
        check(lib().sch_synth_obs(self._h, _ptr(u), seed, ctr, _ptr(y), _stream()), "sch_synth_obs")
        return y

    def diagnostics(self, u: torch.Tensor, u_truth: torch.Tensor, ws: Optional[torch.Tensor] = None,
                    out: Optional[torch.Tensor] = None):
        """[EMRE, RB, RES, RMSE, scratch x4] (double, on the device)."""
        N = u.shape[0]
        _need(u, self.dtype, (N, self.n), "u")
        _need(u_truth, self.dtype, (self.n,), "u_truth")
        ws = torch.empty(self.n, dtype=torch.float64, device=u.device) if ws is None else ws
        out = torch.empty(8, dtype=torch.float64, device=u.device) if out is None else out
        check(lib().pf_diagnostics(self._h, N, _ptr(u), _ptr(u_truth), _ptr(ws), _ptr(out), _stream()),
              "pf_diagnostics")
        return out

    def adjoint_window(self, m_start: torch.Tensor, dW: torch.Tensor, lam: Optional[torch.Tensor],
                       y: torch.Tensor, ckpt: Optional[int] = None, want_dW: bool = True, want_m0: bool = True,
                       ws: Optional[torch.Tensor] = None):
        """sch_adjoint_window: J and its gradients for every particle.  ckpt: the
        checkpoint interval; None keeps every state of the window from the forward
        pass (one segment, nothing recomputed), a smaller interval trades
        recomputation for workspace."""
        N, nsteps, K = dW.shape
        ckpt = _ckpt(ckpt, nsteps)
        _need(m_start, self.dtype, (N, self.n), "m_start")
        _need(dW, self.dtype, (N, nsteps, self.K), "dW")
        _need(y, self.dtype, (self.M,), "y")
        if lam is not None:
            _need(lam, self.dtype, (N, nsteps, self.K), "lambda")
        dev = dW.device
        J = torch.empty(N, dtype=torch.float64, device=dev)
        g_lam = torch.empty_like(dW)
        g_dW = torch.empty_like(dW) if want_dW else None
        g_m0 = torch.empty_like(m_start) if want_m0 else None
        iters = torch.empty(N, dtype=torch.int32, device=dev)
        status = torch.empty(N, dtype=torch.int32, device=dev)
        need = int(lib().sch_adjoint_workspace_bytes(self._h, N, nsteps, ckpt))
        if ws is None:
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
        check(lib().sch_adjoint_window(self._h, N, nsteps, ckpt, _ptr(m_start), _ptr(dW), _ptr(lam), _ptr(y),
                                       _ptr(J), _ptr(g_lam), _ptr(g_dW), _ptr(g_m0), _ptr(iters), _ptr(status),
                                       _ptr(ws), ws.numel() * ws.element_size(), _stream()), "sch_adjoint_window")
        return dict(J=J, g_lam=g_lam, g_dW=g_dW, g_m0=g_m0, iters=iters, status=status)

    def adjoint_workspace_bytes(self, N: int, nsteps: int, ckpt: Optional[int] = None) -> int:
        """Bytes of the workspace sch_adjoint_window needs for N particles."""
        return int(lib().sch_adjoint_workspace_bytes(self._h, N, nsteps, _ckpt(ckpt, nsteps)))

    def mala_jitter(self, m_start: torch.Tensor, dW: torch.Tensor, lam: Optional[torch.Tensor], y: torch.Tensor,
                    theta: float, h: float, n_iter: int, seed: int, ctr: int, particle0: int = 0,
                    ckpt: Optional[int] = None):
        """n_iter MALA moves of every particle's window noise at temperature theta, updating dW in
        place: pf_mala_propose, sch_adjoint_window at the proposal, pf_mala_accept (iteration j
        keyed ctr + j).  The window is then run once at the final noise.
        Returns dict(accepts, m, u, nll, logG, status)."""
        N, nsteps, K = dW.shape
        _need(dW, self.dtype, (N, nsteps, self.K), "dW")
        ws = torch.empty(self.adjoint_workspace_bytes(N, nsteps, ckpt), dtype=torch.uint8, device=dW.device)
        cur = self.adjoint_window(m_start, dW, lam, y, ckpt=ckpt, want_m0=False, ws=ws)
        J, gJ = cur["J"], cur["g_dW"]
        dWp = torch.empty_like(dW)
        acc = torch.zeros(N, dtype=torch.int32, device=dW.device)
        for j in range(n_iter):
            self.mala_propose(dW, lam, gJ, dWp, theta, h, seed, ctr + j, particle0)
            prop = self.adjoint_window(m_start, dWp, lam, y, ckpt=ckpt, want_m0=False, ws=ws)
            self.mala_accept(dW, dWp, lam, J, prop["J"], gJ, prop["g_dW"], acc, theta, h, seed, ctr + j, particle0)
        fin = self.ensemble_step(m_start, dW, lam, y)
        return dict(accepts=acc, m=fin["m"], u=fin["u"], nll=fin["nll"], logG=fin["logG"], status=fin["status"])

    def mala_propose(self, dW: torch.Tensor, lam: Optional[torch.Tensor], gJ: torch.Tensor, dW_prop: torch.Tensor,
                     theta: float, h: float, seed: int, ctr: int, particle0: int = 0) -> None:
        """pf_mala_propose: dW_prop = dW - (h/2) dt grad U(dW) + sqrt(h dt) z."""
        N, nsteps, _ = dW.shape
        check(lib().pf_mala_propose(self._h, N, nsteps, theta, h, seed, ctr, particle0, _ptr(dW), _ptr(lam),
                                    _ptr(gJ), _ptr(dW_prop), _stream()), "pf_mala_propose")

    def mala_accept(self, dW: torch.Tensor, dW_prop: torch.Tensor, lam: Optional[torch.Tensor], J: torch.Tensor,
                    J_prop: torch.Tensor, gJ: torch.Tensor, gJ_prop: torch.Tensor, accepts: Optional[torch.Tensor],
                    theta: float, h: float, seed: int, ctr: int, particle0: int = 0) -> None:
        """pf_mala_accept: the Metropolis-Hastings decision; accepted rows of dW, J, gJ take the proposal's."""
        N, nsteps, _ = dW.shape
        check(lib().pf_mala_accept(self._h, N, nsteps, theta, h, seed, ctr, particle0, _ptr(dW), _ptr(dW_prop),
                                   _ptr(lam), _ptr(J), _ptr(J_prop), _ptr(gJ), _ptr(gJ_prop), _ptr(accepts),
                                   _stream()), "pf_mala_accept")

    def nudge(self, m_start: torch.Tensor, y: torch.Tensor, nsteps: int, mode: str = "sequential",
              max_iter: int = 50, gtol: float = 1e-8, ckpt: Optional[int] = None, seed: int = 0, ctr: int = 0,
              lam0: Optional[torch.Tensor] = None, ws: Optional[torch.Tensor] = None):
        """pf_nudge: L-BFGS nudging drifts and the revealed increments for every particle
        (ckpt as in adjoint_window)."""
        N = m_start.shape[0]
        ckpt = _ckpt(ckpt, nsteps)
        _need(m_start, self.dtype, (N, self.n), "m_start")
        _need(y, self.dtype, (self.M,), "y")
        dev = m_start.device
        lam = torch.zeros((N, nsteps, self.K), dtype=self.dtype, device=dev) if lam0 is None else lam0.clone()
        _need(lam, self.dtype, (N, nsteps, self.K), "lambda")
        dW = torch.empty_like(lam)
        J = torch.empty(N, dtype=torch.float64, device=dev)
        iters = torch.empty(N, dtype=torch.int32, device=dev)
        status = torch.empty(N, dtype=torch.int32, device=dev)
        need = int(lib().pf_nudge_workspace_bytes(self._h, N, nsteps, ckpt))
        if ws is None:
            ws = torch.empty(need, dtype=torch.uint8, device=dev)
        m = {"sequential": 0, "open_loop": 1}[mode]
        check(lib().pf_nudge(self._h, N, nsteps, m, max_iter, gtol, ckpt, seed, ctr, _ptr(m_start), _ptr(y),
                             _ptr(lam), _ptr(dW), _ptr(J), _ptr(iters), _ptr(status), _ptr(ws),
                             ws.numel() * ws.element_size(), _stream()), "pf_nudge")
        return dict(lam=lam, dW=dW, J=J, iters=iters, status=status)

    def prior_sample(self, N: int, u_truth: torch.Tensor, seed: int, scale: float):
        _need(u_truth, self.dtype, (self.n,), "u_truth")
        m = torch.empty((N, self.n), dtype=self.dtype, device="cuda")
        u = torch.empty_like(m)
        check(lib().sch_prior_sample(self._h, N, _ptr(u_truth), seed, scale, _ptr(m), _ptr(u), _stream()),
              "sch_prior_sample")
        return m, u

    def prior_exp1(self, N: int, seed: int, particle0: int = 0):
        """sch_prior_exp1: members particle0 .. particle0 + N - 1 of the Exp 1 initial ensemble."""
        m = torch.empty((N, self.n), dtype=self.dtype, device="cuda")
        u = torch.empty_like(m)
        check(lib().sch_prior_exp1(self._h, N, seed, particle0, _ptr(m), _ptr(u), _stream()), "sch_prior_exp1")
        return m, u


# ---------------------------------------------------------------------- #
# filter entry points that need no model context
# ---------------------------------------------------------------------- #
def pf_temper(nll: torch.Tensor, logG: Optional[torch.Tensor], theta: float, ess_min: float,
              wbar: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None, mode: str = "largest"):
    """Returns (wbar, out) with out = [dtheta, ESS, theta_new, ESS of the whole remaining step]
    on the device; phi = nll - logG.  mode "largest": the largest passing dtheta
    (pf_temper); "halving": the first passing (1 - theta) 2^-k (pf_temper_halving)."""
    N = nll.shape[0]
    _need(nll, torch.float64, (N,), "nll")
    if logG is not None:
        _need(logG, torch.float64, (N,), "logG")
    wbar = torch.empty_like(nll) if wbar is None else wbar
    out = torch.empty(4, dtype=torch.float64, device=nll.device) if out is None else out
    fn = {"largest": lib().pf_temper, "halving": lib().pf_temper_halving}[mode]
    check(fn(N, _ptr(nll), _ptr(logG), theta, ess_min, _ptr(wbar), _ptr(out), _stream()), "pf_temper")
    return wbar, out


def pf_resample(wbar: torch.Tensor, seed: int, stage_ctr: int, arrays: Sequence[torch.Tensor] = (),
                ws: Optional[torch.Tensor] = None, idx: Optional[torch.Tensor] = None):
    """Offspring indices (int32 [N]); gathers each tensor of ``arrays`` in place through ``ws``."""
    N = wbar.shape[0]
    _need(wbar, torch.float64, (N,), "wbar")
    idx = torch.empty(N, dtype=torch.int32, device=wbar.device) if idx is None else idx
    na = len(arrays)
    ptrs = (ct.c_void_p * max(na, 1))(*[a.data_ptr() for a in arrays])
    rows = (ct.c_size_t * max(na, 1))(*[a[0].numel() * a.element_size() for a in arrays])
    for a in arrays:
        if a.shape[0] != N or not a.is_contiguous():
            raise ValueError("arrays must be contiguous with N rows")
    total = sum(rows[i] for i in range(na))
    if na and ws is None:
        ws = torch.empty(N * total, dtype=torch.uint8, device=wbar.device)
    ws_bytes = 0 if ws is None else ws.numel() * ws.element_size()
    check(lib().pf_resample(N, _ptr(wbar), seed, stage_ctr, _ptr(idx), na, ptrs if na else None,
                            rows if na else None, _ptr(ws), ws_bytes, _stream()), "pf_resample")
    return idx


def pf_resample_static(wbar: torch.Tensor, seed: int, stage_ctr: int, arrays: Sequence[torch.Tensor] = (),
                       idx: Optional[torch.Tensor] = None):
    """As pf_resample, but the in-place gathers are staged in the library's own
    device scratch (no allocation, no workspace argument; each array at most
    PF_RESAMPLE_STATIC_BYTES).  Calls that overlap on the GPU share that scratch."""
    N = wbar.shape[0]
    _need(wbar, torch.float64, (N,), "wbar")
    idx = torch.empty(N, dtype=torch.int32, device=wbar.device) if idx is None else idx
    na = len(arrays)
    for a in arrays:
        if a.shape[0] != N or not a.is_contiguous():
            raise ValueError("arrays must be contiguous with N rows")
    ptrs = (ct.c_void_p * max(na, 1))(*[a.data_ptr() for a in arrays])
    rows = (ct.c_size_t * max(na, 1))(*[a[0].numel() * a.element_size() for a in arrays])
    check(lib().pf_resample_static(N, _ptr(wbar), seed, stage_ctr, _ptr(idx), na, ptrs if na else None,
                                   rows if na else None, _stream()), "pf_resample_static")
    return idx


def pf_temper_dev(nll: torch.Tensor, logG: Optional[torch.Tensor], theta_dev: torch.Tensor, ess_min: float,
                  wbar: torch.Tensor, out: torch.Tensor, mode: str = "largest"):
    """Device-gated tempering stage: theta read from the device scalar theta_dev; writes
    out[5] = [dtheta, ESS, theta_new, ESS of the whole remaining step, active]."""
    N = nll.shape[0]
    _need(nll, torch.float64, (N,), "nll")
    _need(out, torch.float64, (5,), "out")
    md = {"largest": 0, "halving": 1}[mode]
    check(lib().pf_temper_dev(N, _ptr(nll), _ptr(logG), _ptr(theta_dev), ess_min, md, _ptr(wbar), _ptr(out),
                              _stream()), "pf_temper_dev")
    return wbar, out


def pf_resample_gated(wbar: torch.Tensor, seed: int, stage_ctr: int, gate: torch.Tensor, idx: torch.Tensor):
    """Offspring indices of a device-gated stage (identity when *gate == 0)."""
    N = wbar.shape[0]
    check(lib().pf_resample_gated(N, _ptr(wbar), seed, stage_ctr, _ptr(gate), _ptr(idx), _stream()),
          "pf_resample_gated")
    return idx


def pf_gather_rows(idx: torch.Tensor, src: torch.Tensor, dst: torch.Tensor):
    N = idx.shape[0]
    row = src[0].numel() * src.element_size()
    check(lib().pf_gather_rows(N, _ptr(idx), _ptr(src), _ptr(dst), row, _stream()), "pf_gather_rows")
    return dst


def pf_resample_workspace_bytes(N: int, row_bytes_total: int) -> int:
    return int(lib().pf_resample_workspace_bytes(N, row_bytes_total))


def _ckpt(ckpt: Optional[int], nsteps: int) -> int:
    """The adjoint's checkpoint interval: None is the whole window (every state kept)."""
    return max(1, nsteps) if ckpt is None else ckpt


class NudgingCost(torch.autograd.Function):
    """J(m_start, dW, lambda) = NLL(u_end) + 1/2 dt sum lambda^2 per particle, with the
    hand-written adjoint (sch_adjoint_window) as its backward.

    forward(model, m_start, dW, lam, y, ckpt) -> J [N] (double).  The backward
    returns the adjoint's gradients, scaled per particle by the incoming
    gradient of J (autograd's chain rule).
    """

    @staticmethod
    def forward(ctx, model: SchModel, m_start, dW, lam, y, ckpt: Optional[int] = None):
        out = model.adjoint_window(m_start.contiguous(), dW.contiguous(), lam.contiguous(), y.contiguous(), ckpt)
        ctx.save_for_backward(out["g_m0"], out["g_dW"], out["g_lam"])
        return out["J"]

    @staticmethod
    def backward(ctx, gJ):
        g_m0, g_dW, g_lam = ctx.saved_tensors
        s = gJ.to(g_lam.dtype)
        return (None, g_m0 * s[:, None], g_dW * s[:, None, None], g_lam * s[:, None, None], None, None)


class ProposalNet:
    """Learned drift proposal (nn_forward / nn_backward / nn_adam_step).

    ``params`` is the flat FP32 parameter vector in the library's layout
    (per layer w[C][Cin][5], b[C]; then Wh[K Ns][C K], bh[K Ns]); when omitted
    it is initialised with a seeded He-normal draw.  ``precision`` is "fp32" (FP32
    contractions on the CUDA cores) or "bf16" (BF16 operands, FP32 accumulation, on the
    tensor cores); it can be changed later with ``set_precision``.
    """

    def __init__(self, n: int, K: int, Ns: int, M: int, sigma: float, C: int = 64,
                 params: Optional[torch.Tensor] = None, seed: int = 0, precision: str = "fp32"):
        self.shape = NNShape(n, K, Ns, C, M, sigma, self._prec(precision))
        self.precision = precision
        self.n, self.K, self.Ns, self.C, self.M = n, K, Ns, C, M
        self.count = int(lib().nn_param_count(ct.byref(self.shape)))
        if self.count == 0:
            raise ValueError("invalid network shape")
        if params is None:
            g = torch.Generator(device="cpu").manual_seed(seed)
            parts, cin = [], 2
            for _ in range(4):
                parts.append(torch.randn(C * cin * 5, generator=g) * (2.0 / (cin * 5)) ** 0.5)
                parts.append(torch.zeros(C))
                cin = C
            parts.append(torch.randn(K * Ns * C * K, generator=g) * (1.0 / (C * K)) ** 0.5)
            parts.append(torch.zeros(K * Ns))
            params = torch.cat(parts)
        self.params = params.to(device="cuda", dtype=torch.float32).contiguous()
        if self.params.numel() != self.count:
            raise ValueError(f"expected {self.count} parameters")
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        self._ws = None

    @staticmethod
    def _prec(precision: str) -> int:
        return {"fp32": _lib.NN_FP32, "bf16": _lib.NN_BF16}[precision]

    def set_precision(self, precision: str) -> None:
        """Switch the contractions between FP32 ("fp32") and BF16 with FP32 accumulation ("bf16")."""
        self.shape.precision = self._prec(precision)
        self.precision = precision

    def _workspace(self, B: int):
        need = int(lib().nn_workspace_bytes(ct.byref(self.shape), B))
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        return self._ws

    def forward(self, u_start: torch.Tensor, y: torch.Tensor, out: Optional[torch.Tensor] = None):
        """lambda [B, Ns, K] for velocities [B, n]; y is [M] (shared) or [B, M]."""
        B = u_start.shape[0]
        _need(u_start, torch.float32, (B, self.n), "u_start")
        ys = 0 if y.dim() == 1 else self.M
        out = torch.empty((B, self.Ns, self.K), dtype=torch.float32, device="cuda") if out is None else out
        ws = self._workspace(B)
        check(lib().nn_forward(ct.byref(self.shape), B, _ptr(self.params), _ptr(u_start), _ptr(y), ys, _ptr(out),
                               _ptr(ws), ws.numel(), _stream()), "nn_forward")
        return out

    def loss_and_grad(self, u_start: torch.Tensor, y: torch.Tensor, target: torch.Tensor):
        B = u_start.shape[0]
        _need(u_start, torch.float32, (B, self.n), "u_start")
        _need(target, torch.float32, (B, self.Ns, self.K), "target")
        ys = 0 if y.dim() == 1 else self.M
        grads = torch.empty_like(self.params)
        loss = torch.empty(1, dtype=torch.float64, device="cuda")
        ws = self._workspace(B)
        check(lib().nn_backward(ct.byref(self.shape), B, _ptr(self.params), _ptr(u_start), _ptr(y), ys,
                                _ptr(target), _ptr(grads), _ptr(loss), _ptr(ws), ws.numel(), _stream()),
              "nn_backward")
        return loss, grads

    def adam_step(self, grads: torch.Tensor, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999,
                  eps: float = 1e-8):
        self.t += 1
        check(lib().nn_adam_step(self.count, _ptr(self.params), _ptr(grads), _ptr(self.m), _ptr(self.v), self.t,
                                 lr, b1, b2, eps, _stream()), "nn_adam_step")

    def train_step(self, u_start, y, target, lr: float = 1e-3):
        loss, grads = self.loss_and_grad(u_start, y, target)
        self.adam_step(grads, lr)
        return loss
