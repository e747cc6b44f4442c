"""FP64 oracle of the nudging optimisation (test infrastructure only).

Sec. 3.1.3 of the paper: a drift lambda added to the noise (the nudged SDE)
is chosen per particle to make the observations likely, and the Girsanov
factor corrects the weight.  For a window of Ns steps the cost of a drift is

    J(lambda) = NLL(u_end) + 1/2 sum_{n,k} (lambda_k^n)^2 dt

(the negative log of W~ = W G with the drawn increments of the steps still
to come set to zero, so that the lambda dW term of log G vanishes for them).
Two schedules:

* ``nudge_sequential``: the paper's adapted scheme -- for n = 0..Ns-1,
  optimise lambda^n with all later increments and drifts zero, then draw the
  increment dW^n ~ N(0, dt) (Philox, purpose TAG_NUDGE);
* ``nudge_open_loop``: optimise all lambda at once with every dW = 0, then
  draw all increments (lambda depends on no noise, so it is adapted).

Gradients come from the forward tangent-linear model: for each step the
implicit relation R(m1; m0, dU) = 0 of Eq. fde1 is differentiated with dense
Jacobians, dm1 = -J1^{-1} (J0 dm0 + B ddU), and all K Ns drift directions are
carried forward at once.  This is independent of the reverse-mode adjoint of
the CUDA path.  The optimiser is scipy's L-BFGS-B.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize

from oracle import filter as _F
from oracle import rng as _rng


def obs_grad_u(u_end: np.ndarray, y: np.ndarray, sigma: float) -> np.ndarray:
    """d NLL / d u_end: (u(x_j) - y_j) / sigma^2 at the observed nodes, zero elsewhere."""
    n = len(u_end)
    y = np.asarray(y, dtype=np.float64)
    obs = _F.observed(y)
    idx = _F.obs_indices(n, len(y))[obs]
    g = np.zeros(n)
    g[idx] = (u_end[idx] - y[obs]) / sigma ** 2
    return g


def dense_ops(model):
    Md = model.dense(model.mass())
    Kd = model.dense(model.stiffness())
    Hd = model.dense(model.helmholtz())
    HinvM = np.linalg.solve(Hd, Md)
    return Md, Kd, HinvM


def advection_in_v(model, mbar: np.ndarray) -> np.ndarray:
    """Dense matrix of the linear map v -> A(mbar, v), assembled column by column (linearity)."""
    n = model.n
    B = np.empty((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[:] = 0.0
        e[j] = 1.0
        B[:, j] = model.apply(model.advection(e), mbar)
    return B


def step_jacobians(model, m0, m1, dU, ops=None):
    """J1 = dR/dm1, J0 = dR/dm0 and B = dR/d(dU) of R = M (m1 - m0) + mu dt K mbar + A(mbar, dv)."""
    Md, Kd, HinvM = dense_ops(model) if ops is None else ops
    u0 = model.u_from_m(m0)
    u1 = model.u_from_m(m1)
    mbar = 0.5 * (m0 + m1)
    dv = 0.5 * model.dt * (u0 + u1) + dU
    Av = model.dense(model.advection(dv))
    Bm = advection_in_v(model, mbar)
    common = 0.5 * model.mu * model.dt * Kd + 0.5 * Av + Bm @ (0.5 * model.dt * HinvM)
    return Md + common, -Md + common, Bm


def cost(model, m0, dW, lam, y, sigma) -> float:
    """J = NLL(u_end) + 1/2 sum lambda^2 dt for one particle."""
    _, u_end, _, _ = model.window(m0, dW, lam)
    return float(_F.nll(u_end[None], y, sigma)[0] + 0.5 * model.dt * np.sum(np.asarray(lam) ** 2))


def cost_and_gradient(model, m0, dW, lam, y, sigma, var_steps=None):
    """J and dJ/dlambda over the steps in ``var_steps`` (default: all), by tangent linearisation.

    Returns (J, grad) with grad of shape [len(var_steps), K].
    """
    dW = np.asarray(dW, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    Ns, K = dW.shape          # K: Brownian motions per step (the Matern noise: one per cell)
    var_steps = list(range(Ns)) if var_steps is None else list(var_steps)
    col = {s: i for i, s in enumerate(var_steps)}
    nvar = len(var_steps) * K
    _, u_end, _, _, traj = model.window(m0, dW, lam, return_traj=True)
    ops = dense_ops(model)
    Xi = model.noise_matrix()                 # d dU / d(dW + lambda dt): [n, K]
    D = np.zeros((model.n, nvar))             # d m_s / d lambda
    for s in range(Ns):
        m_s, m_s1 = traj[s][0], traj[s + 1][0]
        dU = model.noise(dW[s], lam[s])
        J1, J0, Bm = step_jacobians(model, m_s, m_s1, dU, ops)
        rhs = J0 @ D
        if s in col:
            c = col[s]
            rhs[:, c * K:(c + 1) * K] += Bm @ (model.dt * Xi)
        D = -np.linalg.solve(J1, rhs)
    du = ops[2] @ D
    g_u = obs_grad_u(u_end, y, sigma)
    grad = (g_u @ du).reshape(len(var_steps), K) + model.dt * lam[var_steps]
    J = float(_F.nll(u_end[None], y, sigma)[0] + 0.5 * model.dt * np.sum(lam ** 2))
    return J, grad


def _minimise(fun_grad, x0, maxiter, gtol):
    res = minimize(fun_grad, x0, jac=True, method="L-BFGS-B",
                   options=dict(maxiter=maxiter, gtol=gtol, ftol=0.0, maxcor=10))
    return res.x, res


def nudge_open_loop(model, m0, y, sigma, Ns, K, maxiter=200, gtol=1e-10, lam0=None):
    """All drifts at once with every increment zero. Returns (lambda [Ns, K], scipy result)."""
    dW0 = np.zeros((Ns, K))

    def fg(x):
        lam = x.reshape(Ns, K)
        J, g = cost_and_gradient(model, m0, dW0, lam, y, sigma)
        return J, g.ravel()

    x0 = np.zeros(Ns * K) if lam0 is None else np.asarray(lam0, dtype=np.float64).ravel()
    x, res = _minimise(fg, x0, maxiter, gtol)
    return x.reshape(Ns, K), res


def nudge_sequential(model, m0, y, sigma, Ns, K, seed, particle, ctr, maxiter=100, gtol=1e-10):
    """The adapted schedule of Sec. 3.1.3.

    For n = 0..Ns-1: optimise lambda^n with dW^{>=n} = 0 and lambda^{>n} = 0,
    then reveal dW^n = sqrt(dt) z, z keyed (seed, TAG_NUDGE, (k / 4, n, particle, ctr)).
    Returns (lambda [Ns, K], dW [Ns, K]).
    """
    lam = np.zeros((Ns, K))
    dW = np.zeros((Ns, K))
    z = _rng.normals(seed, _rng.TAG_NUDGE, K, np.arange(Ns, dtype=np.uint64), np.uint64(particle),
                     np.uint64(ctr))
    for n in range(Ns):
        def fg(x, n=n):
            lam_try = lam.copy()
            lam_try[n] = x
            J, g = cost_and_gradient(model, m0, dW, lam_try, y, sigma, var_steps=[n])
            return J, g.ravel()

        x, _ = _minimise(fg, np.zeros(K), maxiter, gtol)
        lam[n] = x
        dW[n] = np.sqrt(model.dt) * z[n]
    return lam, dW
