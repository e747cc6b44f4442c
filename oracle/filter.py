"""FP64 oracle of the particle-filter steps (test infrastructure only).

Sec. 3 of the paper: likelihood weights (Eq. loglikeq), effective sample size
(Eq. ess), adaptive tempering (Sec. 3.1.2), systematic resampling
(Sec. 3.1.1, Gordon et al. 1993), PCN jittering of the noise increments
(Sec. 3.1.2), the discrete Girsanov weight of a nudged path
(Eq. girsanov DG approx), the diagnostics EMRE, RB, RES (Sec. 4.1.1) and a
MALA jitter on the PCN jitter's target (the gradient-informed move Sec. 5
lists as future work; preconditioner C = dt, the prior covariance of dW).

Readings of the text that the code fixes:
* observation points are the M distinct nodes x_j = j L / M, j = 0..M-1; an
  entry of y that is NaN is not observed;
* the Girsanov log-weight of increments dW drawn under drift lambda is
  logG = -sum_{n<Ns} sum_k (lambda_k^n dW_k^n + 1/2 (lambda_k^n)^2 dt), the
  ratio of the N(0, dt) prior density to the proposal density of the increment
  actually applied (dW + lambda dt); "W~ = W + G" is addition of logs;
* the negative log-weight of a particle is phi = NLL - logG (= -log W~);
* tempering keeps the largest dtheta in (0, 1 - theta] whose tempered weights
  exp(-dtheta phi) have ESS >= N*, by 60 bisection steps on [0, 1 - theta];
* PCN accepts with probability min(1, exp(w0 - w1)), w = theta phi (the
  theta-adjusted weight with W replaced by W~);
* systematic resampling runs on exact integers (see ``systematic_resample``).
"""
from __future__ import annotations

import math

import numpy as np

from oracle import rng as _rng


# ---------------------------------------------------------------------- #
# weights
# ---------------------------------------------------------------------- #
def obs_indices(n: int, M: int) -> np.ndarray:
    """Node indices of the M observation points x_j = j L / M."""
    return np.arange(M) * (n // M)


def observed(y: np.ndarray) -> np.ndarray:
    """Mask of the observed points: an entry of y that is NaN is not observed (Exp 2
    of Sec. 4 observes only [0, L/2])."""
    return ~np.isnan(np.asarray(y, dtype=np.float64))


def nll(u: np.ndarray, y: np.ndarray, sigma: float) -> np.ndarray:
    """Negative log of Eq. loglikeq: 1/2 sum_j ((u(x_j) - y_j) / sigma)^2 for each particle,
    over the observed points j (y_j not NaN)."""
    u = np.atleast_2d(np.asarray(u, dtype=np.float64))
    y = np.asarray(y, dtype=np.float64)
    M = len(y)
    obs = observed(y)
    idx = obs_indices(u.shape[1], M)[obs]
    r = (u[:, idx] - y[obs][None, :]) / sigma
    return 0.5 * np.sum(r * r, axis=1)


def girsanov_logG(lam: np.ndarray, dW: np.ndarray, dt: float) -> np.ndarray:
    """log G = -sum_n sum_k (lambda dW + 1/2 lambda^2 dt) per particle (Eq. girsanov DG approx)."""
    lam = np.asarray(lam, dtype=np.float64)
    dW = np.asarray(dW, dtype=np.float64)
    axes = tuple(range(1, lam.ndim))
    return -np.sum(lam * dW + 0.5 * lam * lam * dt, axis=axes)


def normalise(logw: np.ndarray) -> np.ndarray:
    """w_bar = w / sum w from log-weights, shifted by the maximum."""
    lw = np.asarray(logw, dtype=np.float64)
    w = np.exp(lw - np.max(lw))
    return w / np.sum(w)


def ess(logw: np.ndarray) -> float:
    """Eq. ess: ESS = 1 / sum w_bar^2."""
    wb = normalise(logw)
    return float(1.0 / np.sum(wb * wb))


def temper(phi: np.ndarray, theta: float, ess_min: float, iters: int = 60, mode: str = "largest"):
    """Adaptive tempering step (Sec. 3.1.2).

    mode "largest": the largest dtheta in (0, 1 - theta] with
    ESS(exp(-dtheta phi)) >= ess_min.  If the whole remaining step passes it is
    taken; otherwise bisection on [0, 1 - theta] for ``iters`` steps keeps the
    largest passing point.  mode "halving": the first of (1 - theta) 2^-k,
    k = 0 .. iters, that passes.  In both, if even the smallest point tried
    fails (only possible for astronomically spread phi), the smallest point
    tried is returned, so tempering always advances.  Returns (dtheta, w_bar at
    dtheta, ESS at dtheta).
    """
    phi = np.asarray(phi, dtype=np.float64)
    rest = 1.0 - theta
    if ess(-rest * phi) >= ess_min:
        d = rest
    elif mode == "halving":
        # Sec. 3.1.2 read literally ("repeatedly reduces dtheta until the condition
        # holds"): the first of rest 2^-k, k = 1 .. iters, that passes, else the last tried
        for k in range(1, iters + 1):
            d = rest * 2.0 ** -k
            if ess(-d * phi) >= ess_min:
                break
    else:
        lo, hi = 0.0, rest
        for _ in range(iters):
            mid = 0.5 * (lo + hi)
            if ess(-mid * phi) >= ess_min:
                lo = mid
            else:
                hi = mid
        d = lo if lo > 0.0 else hi
    return d, normalise(-d * phi), ess(-d * phi)


# ---------------------------------------------------------------------- #
# systematic resampling on integers
# ---------------------------------------------------------------------- #
RESAMPLE_QBITS = 50
RESAMPLE_UBITS = 53


def systematic_resample(wbar: np.ndarray, u53: int) -> np.ndarray:
    """Systematic resampling (Gordon et al. 1993) in exact integer arithmetic.

    Quantise q_i = floor(w_bar_i 2^50), T = sum q, C_j = q_0 + .. + q_j.
    Slot i takes the smallest j with C_j > floor((i 2^53 + U) T / (N 2^53)),
    U = u53 in [0, 2^53): the positions (i + U 2^-53) / N of systematic
    resampling, scaled to the integer total T.  Every value is an integer, so
    the offspring indices do not depend on the summation order.
    """
    wbar = np.asarray(wbar, dtype=np.float64)
    N = len(wbar)
    q = [int(math.floor(float(w) * 2.0 ** RESAMPLE_QBITS)) for w in wbar]
    if any(v < 0 for v in q):
        raise ValueError("negative weight")
    C = []
    acc = 0
    for v in q:
        acc += v
        C.append(acc)
    T = acc
    if T == 0:
        raise ValueError("all quantised weights are zero")
    idx = np.empty(N, dtype=np.int64)
    scale = N << RESAMPLE_UBITS
    j = 0
    for i in range(N):
        t = ((i << RESAMPLE_UBITS) + int(u53)) * T // scale
        while C[j] <= t:
            j += 1
        idx[i] = j
    return idx


def resample_offset(seed: int, stage_ctr: int) -> int:
    return _rng.u53_int(seed, _rng.TAG_RESAMPLE, stage_ctr)


# ---------------------------------------------------------------------- #
# PCN jittering
# ---------------------------------------------------------------------- #
def pcn_rho(delta: float) -> float:
    """rho = (2 - delta) / (2 + delta); then sqrt(1 - rho^2) = sqrt(8 delta) / (2 + delta)."""
    return (2.0 - delta) / (2.0 + delta)


def pcn_propose(dW: np.ndarray, dW_hat: np.ndarray, rho: float) -> np.ndarray:
    """dW -> rho dW + sqrt(1 - rho^2) dW_hat, dW_hat a fresh N(0, dt) draw (Sec. 3.1.2)."""
    return rho * dW + math.sqrt(1.0 - rho * rho) * dW_hat


def jitter(model, m_start, dW, lam, y, sigma, theta, rho, n_iter, seed, ctr, state=None,
           particle0=0, margins=False, gen=_rng.GEN64):
    """n_iter PCN moves of every particle's window noise at temperature theta.

    For iteration j the proposal noise is keyed (seed, TAG_PCN, ctr + j) and the
    accept uniform (seed, TAG_PCN_ACCEPT, ctr + j).  The proposal is run through
    the whole window from m_start; it is accepted iff log U < w0 - w1 with
    w = theta (NLL - logG).  ``state`` = (nll, logG, m_end, u_end) of the
    current noise, recomputed when omitted.
    ``gen``: the generator of the proposal normals (GEN32: the FP32 Matern kernels').
    Returns (dW, nll, logG, m_end, u_end, accepts), and with ``margins`` also the
    [n_iter, N] Metropolis margins (w0 - w1) - log U (a move is accepted iff its
    margin is positive), the [n_iter, N] proposal NLLs and the [n_iter, N] NLLs of the
    current state before each move.
    """
    N, Ns, K = dW.shape
    dW = np.array(dW, dtype=np.float64)
    lam_arr = np.zeros_like(dW) if lam is None else np.asarray(lam, dtype=np.float64)
    if state is None:
        m_end, u_end, _, _ = model.ensemble_window(m_start, dW, lam_arr)
        cur_nll = nll(u_end, y, sigma)
        cur_logG = girsanov_logG(lam_arr, dW, model.dt)
    else:
        cur_nll, cur_logG, m_end, u_end = (np.array(v, dtype=np.float64) for v in state)
    accepts = np.zeros(N, dtype=np.int64)
    marg = np.zeros((n_iter, N))
    prop_nll = np.zeros((n_iter, N))
    prev_nll = np.zeros((n_iter, N))
    for j in range(n_iter):
        hat = _rng.window_increments(seed, _rng.TAG_PCN, N, Ns, K, model.dt, ctr + j, particle0, gen=gen)
        prop = pcn_propose(dW, hat, rho)
        pm, pu, _, _ = model.ensemble_window(m_start, prop, lam_arr)
        p_nll = nll(pu, y, sigma)
        p_logG = girsanov_logG(lam_arr, prop, model.dt)
        w0 = theta * (cur_nll - cur_logG)
        w1 = theta * (p_nll - p_logG)
        pidx = np.arange(particle0, particle0 + N, dtype=np.uint64)
        logU = np.log(_rng.uniform_open0(seed, _rng.TAG_PCN_ACCEPT, pidx, np.uint64(ctr + j)))
        acc = logU < (w0 - w1)
        marg[j] = (w0 - w1) - logU
        prop_nll[j] = p_nll
        prev_nll[j] = cur_nll
        dW[acc] = prop[acc]
        cur_nll[acc] = p_nll[acc]
        cur_logG[acc] = p_logG[acc]
        m_end[acc] = pm[acc]
        u_end[acc] = pu[acc]
        accepts += acc
    if margins:
        return dW, cur_nll, cur_logG, m_end, u_end, accepts, marg, prop_nll, prev_nll
    return dW, cur_nll, cur_logG, m_end, u_end, accepts


# ---------------------------------------------------------------------- #
# MALA jitter: the gradient-informed move Sec. 5 names as future work
# ---------------------------------------------------------------------- #
def mala_step(U, grad_U, x, h, C, z, logu, detail=False):
    """One preconditioned MALA step (Roberts and Tweedie 1996) for the density
    exp(-U): the proposal x' = x - (h/2) C grad U(x) + sqrt(h C) z (C diagonal) is
    accepted iff log u < U(x) - U(x') + log q(x | x') - log q(x' | x), with
    log q(b | a) = -|b - a + (h/2) C grad U(a)|^2_{(h C)^-1} / 2.
    A proposal where U is not finite is rejected.  Returns (x_next, accepted), and
    with ``detail`` also a dict: the margin log alpha - log u, U(x), U(x'), the norms
    of grad U(x), grad U(x') and of the two proposal residuals b - a + (h/2) C grad U(a), and x'.
    """
    x = np.asarray(x, dtype=np.float64)
    C = np.broadcast_to(np.asarray(C, dtype=np.float64), x.shape)
    g = grad_U(x)
    xp = x - 0.5 * h * C * g + np.sqrt(h * C) * z
    gp = grad_U(xp)

    def logq(b, a, ga):
        r = b - a + 0.5 * h * C * ga
        return -0.5 * np.sum(r * r / (h * C))

    log_alpha = U(x) - U(xp) + logq(x, xp, gp) - logq(xp, x, g)
    ok = bool(np.isfinite(U(xp)) and logu < log_alpha)
    if detail:
        info = dict(margin=log_alpha - logu, xp=xp, U0=U(x), U1=U(xp), g=np.linalg.norm(g), gp=np.linalg.norm(gp),
                    rf=np.linalg.norm(xp - x + 0.5 * h * C * g), rb=np.linalg.norm(x - xp + 0.5 * h * C * gp))
        return (xp if ok else x), ok, info
    return (xp if ok else x), ok


def mala_target(model, m_start, dW, lam, y, sigma, theta):
    """U(dW) and grad U for one particle's window noise dW [Ns, K] at temperature theta:
    the PCN jitter's target exp(-theta (NLL - log G)) times the N(0, dt) prior of dW,

        U(dW) = theta (NLL(dW) - log G(dW)) + |dW|^2 / (2 dt).

    With J = NLL + 1/2 dt |lambda|^2, NLL - log G = J + sum lambda dW.  The noise
    applied at a step is dW + lambda dt, so dNLL/ddW = (dNLL/dlambda) / dt, with
    dNLL/dlambda = dJ/dlambda - dt lambda from the tangent-linear model, and
    grad U = theta (dNLL/ddW + lambda) + dW / dt.
    """
    from oracle import nudge as _N
    dt = model.dt
    x = np.asarray(dW, dtype=np.float64)
    la = np.zeros_like(x) if lam is None else np.asarray(lam, dtype=np.float64)
    J, g_lam = _N.cost_and_gradient(model, m_start, x, la, y, sigma)
    U = theta * (J + np.sum(la * x)) + np.sum(x * x) / (2.0 * dt)
    gU = theta * ((g_lam - dt * la) / dt + la) + x / dt
    return U, gU


def mala_jitter(model, m_start, dW, lam, y, sigma, theta, h, n_iter, seed, ctr, particle0=0, margins=False):
    """n_iter MALA moves of every particle's window noise (``mala_target``) with
    preconditioner C = dt (the prior covariance of dW).  For iteration j the
    proposal normals are keyed (seed, TAG_MALA) at counter (k // 4, step,
    particle0 + p, ctr + j) and the accept uniform (seed, TAG_MALA_ACCEPT) at
    (0, 0, particle0 + p, ctr + j).  Returns (dW, nll, logG, accepts), nll and
    logG those of the final noise; with ``margins`` also, per move and particle, the
    ``mala_step`` details with the NLL at both points (NLL = (U - |x|^2 / (2 dt)) /
    theta + log G(x)).
    """
    N, Ns, K = np.shape(dW)
    dt = model.dt
    dW = np.array(dW, dtype=np.float64)
    lam_arr = np.zeros_like(dW) if lam is None else np.asarray(lam, dtype=np.float64)
    accepts = np.zeros(N, dtype=np.int64)
    pidx = np.arange(particle0, particle0 + N, dtype=np.uint64)
    details = []
    for j in range(n_iter):
        z = _rng.window_increments(seed, _rng.TAG_MALA, N, Ns, K, 1.0, ctr + j, particle0)
        logu = np.log(_rng.uniform_open0(seed, _rng.TAG_MALA_ACCEPT, pidx, np.uint64(ctr + j)))
        for p in range(N):
            def U(x, p=p):
                return mala_target(model, m_start[p], x, lam_arr[p], y, sigma, theta)[0]

            def gU(x, p=p):
                return mala_target(model, m_start[p], x, lam_arr[p], y, sigma, theta)[1]

            if margins:
                x0 = dW[p].copy()
                dW[p], ok, info = mala_step(U, gU, x0, h, dt, z[p], logu[p], detail=True)
                x1 = info["xp"]
                for key, xx in (("nll0", x0), ("nll1", x1)):
                    lg = -np.sum(lam_arr[p] * xx + 0.5 * lam_arr[p] ** 2 * dt)
                    Ux = info["U0"] if key == "nll0" else info["U1"]
                    info[key] = (Ux - np.sum(xx * xx) / (2.0 * dt)) / theta + lg
                details.append((j, p, info))
            else:
                dW[p], ok = mala_step(U, gU, dW[p], h, dt, z[p], logu[p])
            accepts[p] += ok
    _, u_end, _, _ = model.ensemble_window(m_start, dW, lam_arr)
    if margins:
        return dW, nll(u_end, y, sigma), girsanov_logG(lam_arr, dW, dt), accepts, details
    return dW, nll(u_end, y, sigma), girsanov_logG(lam_arr, dW, dt), accepts


# ---------------------------------------------------------------------- #
# diagnostics (Sec. 4.1.1)
# ---------------------------------------------------------------------- #
def emre(u_truth, u_ens) -> float:
    """(1/N) sum_n |u_a - u_n| / |u_a| (Euclidean norms over nodes)."""
    ua = np.asarray(u_truth, dtype=np.float64)
    return float(np.mean(np.linalg.norm(u_ens - ua[None, :], axis=1)) / np.linalg.norm(ua))


def rb(u_truth, u_ens) -> float:
    """|u_a - mean_n u_n| / |u_a|."""
    ua = np.asarray(u_truth, dtype=np.float64)
    return float(np.linalg.norm(ua - np.mean(u_ens, axis=0)) / np.linalg.norm(ua))


def res(u_truth, u_ens) -> float:
    """(1/(N-1)) sum_n |u_n - mean u| / |u_a|."""
    ua = np.asarray(u_truth, dtype=np.float64)
    mean = np.mean(u_ens, axis=0)
    N = u_ens.shape[0]
    return float(np.sum(np.linalg.norm(u_ens - mean[None, :], axis=1)) / (N - 1) / np.linalg.norm(ua))


# ---------------------------------------------------------------------- #
# one assimilation cycle (bootstrap forecast, then temper + resample + jitter)
# ---------------------------------------------------------------------- #
def assimilation_cycle(model, m_start, y, sigma, ess_min, rho, n_jitter, seed, cycle,
                       lam=None, dW=None, max_stages=64, temper_mode="largest"):
    """One cycle of Sec. 3.1.2 on the (X_start, dW) representation.

    dW is drawn from (seed, TAG_PRIOR_DW, cycle) unless given.  Stage k tempers
    with the incremental weight exp(-dtheta phi), resamples (X_start, dW, lambda,
    phi) with offset keyed (seed, TAG_RESAMPLE, cycle * 1024 + k), then jitters
    with PCN counters starting at (cycle * 1024 + k) * n_jitter.  Returns a dict
    with the end-of-window state of every particle and per-stage statistics.
    """
    N = m_start.shape[0]
    m_start = np.array(m_start, dtype=np.float64)
    if dW is None:
        raise ValueError("pass dW explicitly (window_increments)")
    dW = np.array(dW, dtype=np.float64)
    Ns = dW.shape[1]
    lam_arr = np.zeros_like(dW) if lam is None else np.array(lam, dtype=np.float64)
    m_end, u_end, iters, _ = model.ensemble_window(m_start, dW, lam_arr)
    cur_nll = nll(u_end, y, sigma)
    cur_logG = girsanov_logG(lam_arr, dW, model.dt)
    theta = 0.0
    stages = []
    k = 0
    while theta < 1.0 and k < max_stages:
        phi = cur_nll - cur_logG
        d, wbar, e = temper(phi, theta, ess_min, mode=temper_mode)
        stage_ctr = cycle * 1024 + k
        idx = systematic_resample(wbar, resample_offset(seed, stage_ctr))
        m_start, dW, lam_arr = m_start[idx], dW[idx], lam_arr[idx]
        cur_nll, cur_logG = cur_nll[idx], cur_logG[idx]
        m_end, u_end = m_end[idx], u_end[idx]
        theta = 1.0 if d >= 1.0 - theta else theta + d
        dW, cur_nll, cur_logG, m_end, u_end, acc = jitter(
            model, m_start, dW, lam_arr, y, sigma, theta, rho, n_jitter, seed,
            stage_ctr * n_jitter, state=(cur_nll, cur_logG, m_end, u_end))
        stages.append(dict(dtheta=d, ess=e, theta=theta, accept_rate=float(acc.sum()) / (N * n_jitter)))
        k += 1
    return dict(m_end=m_end, u_end=u_end, dW=dW, lam=lam_arr, nll=cur_nll, logG=cur_logG,
                stages=stages, Ns=Ns)
