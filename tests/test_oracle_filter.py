"""Pins for the oracle's filter steps (oracle/filter.py).

* ESS (Eq. ess) by brute force and its special cases;
* tempering (Sec. 3.1.2) against a dense scan of dtheta, monotonicity of
  ESS(dtheta) and the stages summing to exactly one;
* systematic resampling (Sec. 3.1.1) against the textbook floating-point
  algorithm, and its defining properties over an enumerated grid of offsets;
* the Girsanov weight (Eq. girsanov DG approx) against the Gaussian density
  ratio it stands for;
* PCN (Sec. 3.1.2): theta = 0 always accepts and keeps N(0, dt) invariant;
  rho = 1 is the identity;
* the tempering + resampling + jittering composition against the exact
  Kalman posterior of a linear-Gaussian toy model.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

from oracle import filter as F
from workloads import random_logweights
from oracle import rng


def test_ess_brute_force():
    r = np.random.default_rng(0)
    for N in range(1, 7):
        lw = r.normal(scale=3, size=N)
        w = [math.exp(v) for v in lw]
        s = sum(w)
        ref = 1.0 / sum((v / s) ** 2 for v in w)
        assert abs(F.ess(lw) - ref) < 1e-12 * ref
    assert abs(F.ess(np.zeros(6)) - 6) < 1e-12
    assert abs(F.ess(np.array([0.0, -1e4, -1e4])) - 1.0) < 1e-12
    assert 1.0 <= F.ess(r.normal(scale=50, size=100)) <= 100


def test_nll_definition_and_girsanov_density_ratio():
    r = np.random.default_rng(1)
    n, M, sigma = 32, 8, 0.05
    u = r.normal(size=(3, n))
    y = r.normal(size=M)
    v = F.nll(u, y, sigma)
    for p in range(3):
        ref = sum(0.5 * ((u[p, j * (n // M)] - y[j]) / sigma) ** 2 for j in range(M))
        assert abs(v[p] - ref) < 1e-12 * ref
    dt = 0.025
    lam = r.normal(size=(2, 5, 4))
    dW = r.normal(scale=math.sqrt(dt), size=(2, 5, 4))
    lg = F.girsanov_logG(lam, dW, dt)
    # prior density of the applied increment over the proposal density of the draw
    sd = math.sqrt(dt)
    ref = (stats.norm.logpdf(dW + lam * dt, scale=sd) - stats.norm.logpdf(dW, scale=sd)).sum(axis=(1, 2))
    assert np.allclose(lg, ref, rtol=1e-12, atol=1e-12)
    assert np.all(F.girsanov_logG(np.zeros_like(lam), dW, dt) == 0.0)


def test_nll_observation_mask():
    # Exp 2 observes [0, L/2] only: entries of y that are NaN are not observed.  The masked
    # NLL is the sum over the observed points alone, written out by hand here.
    r = np.random.default_rng(7)
    n, M, sigma = 64, 16, 0.1
    u = r.normal(size=(2, n))
    y = r.normal(size=M)
    ym = y.copy()
    ym[M // 2 + 1:] = np.nan
    v = F.nll(u, ym, sigma)
    for p in range(2):
        ref = sum(0.5 * ((u[p, j * (n // M)] - y[j]) / sigma) ** 2 for j in range(M // 2 + 1))
        assert abs(v[p] - ref) < 1e-12 * ref
    # nothing observed: likelihood one; every point observed: the unmasked NLL
    assert np.all(F.nll(u, np.full(M, np.nan), sigma) == 0.0)
    assert np.array_equal(F.nll(u, y, sigma), F.nll(u, np.where(F.observed(y), y, np.nan), sigma))
    # a mask that is not a prefix
    ym2 = y.copy()
    ym2[::3] = np.nan
    ref = 0.5 * sum(((u[0, j * (n // M)] - y[j]) / sigma) ** 2 for j in range(M) if j % 3)
    assert abs(F.nll(u, ym2, sigma)[0] - ref) < 1e-12 * ref


def test_temper_against_dense_scan():
    r = np.random.default_rng(2)
    for trial in range(5):
        N = 6
        phi = r.gamma(2.0, 4.0, size=N)
        theta = 0.3 * trial / 5
        ess_min = 3.0
        d, wbar, e = F.temper(phi, theta, ess_min)
        grid = np.linspace(0, 1 - theta, 200001)[1:]
        ok = np.array([F.ess(-g * phi) >= ess_min for g in grid])
        # ESS(dtheta) is non-increasing in dtheta
        assert np.all(np.diff(ok.astype(int)) <= 0)
        if ok.all():
            assert d == 1 - theta
        else:
            last = grid[ok][-1] if ok.any() else 0.0
            step = grid[1] - grid[0]
            assert last - 1e-12 <= d <= last + step
            assert abs(e - ess_min) < 1e-6 * N
        assert np.isclose(wbar.sum(), 1.0)


def test_temper_halving_against_enumeration():
    # halving mode: the first passing point of the sequence (1 - theta) 2^-k, found by
    # enumerating the sequence with the brute-force ESS
    def ess_bf(w):
        w = np.asarray(w, dtype=np.float64)
        return w.sum() ** 2 / (w * w).sum()
    for seed, spread, theta in ((1, 30.0, 0.0), (2, 3.0, 0.4), (3, 300.0, 0.9), (4, 0.001, 0.0)):
        phi = random_logweights(64, seed, spread)
        N = len(phi)
        d, wbar, e = F.temper(phi, theta, 0.5 * N, mode="halving")
        rest = 1.0 - theta
        ks = [k for k in range(61) if ess_bf(np.exp(-rest * 2.0 ** -k * (phi - phi.min()))) >= 0.5 * N]
        assert d == rest * 2.0 ** -(ks[0] if ks else 60)
        assert np.isclose(wbar.sum(), 1.0)
        # never above the largest passing point
        d_big, _, _ = F.temper(phi, theta, 0.5 * N)
        assert d <= d_big * (1 + 1e-12)


def test_temper_stages_sum_to_one():
    r = np.random.default_rng(3)
    phi = r.gamma(2.0, 20.0, size=64)
    theta, n_st = 0.0, 0
    while theta < 1.0:
        d, _, e = F.temper(phi, theta, 32.0)
        assert d > 0 and e >= 32.0 - 1e-9
        theta = 1.0 if d >= 1.0 - theta else theta + d
        n_st += 1
        assert n_st < 100
    assert theta == 1.0 and n_st > 1


def test_resample_matches_float_textbook():
    r = np.random.default_rng(4)
    for N in (1, 2, 5, 64, 1000):
        w = r.gamma(0.5, size=N)
        w /= w.sum()
        u53 = int(r.integers(0, 2**53))
        idx = F.systematic_resample(w, u53)
        U = u53 * 2.0 ** -53
        pos = (np.arange(N) + U) / N
        ref = np.searchsorted(np.cumsum(w), pos, side="right")
        ref = np.minimum(ref, N - 1)
        # the two agree except where a position lies within rounding of a boundary
        c = np.cumsum(w)
        gap = np.min(np.abs(pos[:, None] - c[None, :]), axis=1)
        sel = gap > 1e-12
        assert np.array_equal(idx[sel], ref[sel])
        assert np.all(np.diff(idx) >= 0)


@pytest.mark.parametrize("N", [2, 3, 5, 6])
def test_resample_offspring_counts_over_offsets(N):
    r = np.random.default_rng(10 + N)
    w = r.random(N) ** 3
    w /= w.sum()
    q = np.floor(w * 2.0 ** 50)
    wq = q / q.sum()
    G = 2048
    counts = np.zeros(N)
    for g in range(G):
        u53 = (g * 2**53) // G + 12345
        idx = F.systematic_resample(w, u53)
        cnt = np.bincount(idx, minlength=N)
        assert np.all(cnt >= np.floor(N * wq) - 0) and np.all(cnt <= np.ceil(N * wq))
        counts += cnt
    # mean offspring count over a uniform grid of offsets -> N w_i
    assert np.allclose(counts / G, N * wq, atol=N / G + 1e-12)


def test_resample_degenerate_cases():
    idx = F.systematic_resample(np.array([0.0, 1.0, 0.0]), 0)
    assert list(idx) == [1, 1, 1]
    idx = F.systematic_resample(np.full(4, 0.25), 2**52)
    assert list(idx) == [0, 1, 2, 3]
    with pytest.raises(ValueError):
        F.systematic_resample(np.zeros(3), 0)


def test_pcn_properties():
    dt = 0.025
    r = np.random.default_rng(5)
    x = r.normal(scale=math.sqrt(dt), size=200000)
    hat = r.normal(scale=math.sqrt(dt), size=200000)
    rho = F.pcn_rho(0.15)
    assert abs(math.sqrt(1 - rho * rho) - math.sqrt(8 * 0.15) / 2.15) < 1e-15
    y = F.pcn_propose(x, hat, rho)
    assert abs(y.var() / dt - 1.0) < 0.02 and abs(np.mean(y)) < 0.003
    assert np.corrcoef(x, y)[0, 1] == pytest.approx(rho, abs=0.01)
    assert np.array_equal(F.pcn_propose(x, hat, 1.0), x)


class _RandomWalk:
    """Toy linear-Gaussian model with the oracle model's interface: x_end = x_start + sum dW."""

    dt = 0.025

    def ensemble_window(self, m0, dW, lam=None):
        inc = dW.sum(axis=(1, 2))
        if lam is not None:
            inc = inc + self.dt * lam.sum(axis=(1, 2))
        x = m0[:, 0] + inc
        return x[:, None].copy(), x[:, None].copy(), np.ones((len(x), dW.shape[1]), int), np.ones(len(x), bool)


def test_temper_jitter_matches_kalman():
    # prior x_start ~ N(0, s0^2); x_end = x_start + sum of Ns N(0, dt) increments;
    # y = x_end + N(0, sigma^2).  Exact posterior of x_end is Gaussian.
    N, Ns, s0, sigma, y = 3000, 5, 0.4, 0.1, np.array([0.7])
    model = _RandomWalk()
    r = np.random.default_rng(6)
    m0 = r.normal(scale=s0, size=(N, 1))
    dW = rng.window_increments(11, rng.TAG_PRIOR_DW, N, Ns, 1, model.dt, 0)
    out = F.assimilation_cycle(model, m0, y, sigma, N / 2, 0.9, 10, seed=11, cycle=0, dW=dW)
    prior_var = s0 ** 2 + Ns * model.dt
    post_var = 1.0 / (1.0 / prior_var + 1.0 / sigma ** 2)
    post_mean = post_var * y[0] / sigma ** 2
    x = out["u_end"][:, 0]
    assert len(out["stages"]) > 1
    assert abs(x.mean() - post_mean) < 6 * math.sqrt(post_var / 200)
    assert abs(x.var() / post_var - 1.0) < 0.25


def test_diagnostics():
    ua = np.array([1.0, 2.0, 2.0])
    ens = np.stack([ua, ua])
    assert F.emre(ua, ens) == 0 and F.rb(ua, ens) == 0 and F.res(ua, ens) == 0
    ens = np.stack([ua * 0.5, ua * 1.5])
    assert F.emre(ua, ens) == pytest.approx(0.5)
    assert F.rb(ua, ens) == pytest.approx(0.0, abs=1e-15)
    assert F.res(ua, ens) == pytest.approx(1.0)


def test_mala_step_leaves_a_gaussian_invariant():
    # anisotropic Gaussian target and preconditioner: the chain's moments match the
    # target; without the Metropolis-Hastings correction (or with the proposal
    # ratio inverted) the variances come out biased by 10% or more at this h
    s = np.array([1.0, 2.0])
    C = np.array([1.0, 3.0])

    def U(x):
        return 0.5 * np.sum((x / s) ** 2)

    def gU(x):
        return x / s ** 2

    r = np.random.default_rng(21)
    x = np.zeros(2)
    xs, acc = [], 0
    for _ in range(60000):
        x, ok = F.mala_step(U, gU, x, 0.6, C, r.normal(size=2), np.log(r.uniform()))
        xs.append(x)
        acc += ok
    xs = np.array(xs[2000:])
    assert 0.2 < acc / 60000 < 0.99
    assert np.all(np.abs(xs.mean(axis=0) / s) < 0.05)
    assert np.all(np.abs(xs.var(axis=0) / s ** 2 - 1.0) < 0.05)


def test_mala_step_acceptance_is_the_metropolis_hastings_ratio():
    # log alpha from scipy's Gaussian densities: target pi = N(mu, diag(s^2)) and
    # the proposal kernel N(x - (h/2) C grad U(x), h C)
    mu, s, C, h = np.array([0.3, -1.0, 2.0]), np.array([0.5, 1.5, 1.0]), np.array([0.2, 1.0, 0.7]), 0.9
    U = lambda x: 0.5 * np.sum(((x - mu) / s) ** 2)
    gU = lambda x: (x - mu) / s ** 2
    pi = stats.multivariate_normal(mu, np.diag(s ** 2))
    x, z = np.array([1.0, 0.5, -0.4]), np.array([0.3, -1.2, 0.8])
    xp = x - 0.5 * h * C * gU(x) + np.sqrt(h * C) * z
    q = lambda b, a: stats.multivariate_normal(a - 0.5 * h * C * gU(a), np.diag(h * C)).logpdf(b)
    la = pi.logpdf(xp) - pi.logpdf(x) + q(x, xp) - q(xp, x)
    assert F.mala_step(U, gU, x, h, C, z, la - 1e-9)[1]
    assert not F.mala_step(U, gU, x, h, C, z, la + 1e-9)[1]
    assert np.array_equal(F.mala_step(U, gU, x, h, C, z, la - 1e-9)[0], xp)
    assert np.array_equal(F.mala_step(U, gU, x, h, C, z, la + 1e-9)[0], x)


def test_mala_gradient_of_the_window_target_matches_finite_differences():
    # the gradient mala_target assembles from the tangent-linear dJ/dlambda, with a
    # drift present, against central differences of U built from its definition:
    # theta (NLL - log G) of the window plus the N(0, dt) prior of dW
    from workloads import get_config, random_state, random_increments, random_drift, random_obs
    from tests.helpers import oracle_model
    cfg = get_config("cfg1_f64")
    om = oracle_model(cfg)
    Ns, theta = 3, 0.7
    m0 = om.m_from_u(random_state(cfg, 1, 41)[0])
    dW = random_increments(cfg, 1, 42, steps=Ns)[0]
    la = random_drift(cfg, 1, 43, scale=0.3, steps=Ns)[0]
    y = random_obs(cfg, 44)

    def U_def(x):
        _, u_end, _, _ = om.window(m0, x, la)
        phi = F.nll(u_end[None], y, cfg.sigma)[0] - F.girsanov_logG(la[None], x[None], om.dt)[0]
        return theta * phi + np.sum(x * x) / (2.0 * om.dt)

    U, gU = F.mala_target(om, m0, dW, la, y, cfg.sigma, theta)
    assert U == pytest.approx(U_def(dW), rel=1e-12)
    r = np.random.default_rng(45)
    for _ in range(3):
        d = r.normal(size=dW.shape)
        eps = 1e-4
        fd = (U_def(dW + eps * d) - U_def(dW - eps * d)) / (2 * eps)
        assert np.sum(gU * d) == pytest.approx(fd, rel=1e-6)
