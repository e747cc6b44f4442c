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


def tdev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
