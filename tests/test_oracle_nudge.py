"""Pins for the oracle's nudging cost and tangent-linear gradient (oracle/nudge.py).

* the step Jacobians against central finite differences of the Eq. fde1 residual;
* dJ/dlambda against central finite differences on 16 random directions and a
  second-order Taylor remainder;
* in the linear regime (observations a small perturbation away from the
  un-nudged forecast) the optimiser's drift against the closed-form
  regularised least-squares solution built from a finite-difference Jacobian;
* the sequential schedule reveals exactly the keyed increments and leaves each
  stage at a stationary point.
"""
import math

import numpy as np
import pytest

from oracle import filter as OF
from oracle import nudge as ON
from oracle import rng as ORNG
from oracle.model import Model


def small(n=64, K=4):
    return Model(L=40.0, n=n, alpha=1.0, mu=0.02, dt=0.025, amps=np.full(K // 2, 0.05) / np.arange(1, K // 2 + 1))


def state(m, seed=0):
    r = np.random.default_rng(seed)
    x = m.x
    u = 0.2 / np.cosh(x - 27) + 0.5 / np.cosh(x - 13) + 0.02 * r.normal() * np.sin(2 * np.pi * x / m.L)
    return m.m_from_u(u)


def test_step_jacobians_match_finite_differences():
    m = small(n=32)
    r = np.random.default_rng(1)
    m0 = state(m)
    dU = m.noise(r.normal(scale=0.16, size=m.K), r.normal(size=m.K))
    m1, u1, _, _ = m.step(m0, m.u_from_m(m0), dU)
    J1, J0, B = ON.step_jacobians(m, m0, m1, dU)

    def R(a, b, d):
        return m.residual(a, b, m.u_from_m(a), m.u_from_m(b), d)

    eps = 1e-6
    for j in range(0, m.n, 5):
        e = np.zeros(m.n)
        e[j] = eps
        fd1 = (R(m1 + e, m0, dU) - R(m1 - e, m0, dU)) / (2 * eps)
        fd0 = (R(m1, m0 + e, dU) - R(m1, m0 - e, dU)) / (2 * eps)
        fdb = (R(m1, m0, dU + e) - R(m1, m0, dU - e)) / (2 * eps)
        assert np.allclose(J1[:, j], fd1, atol=1e-8)
        assert np.allclose(J0[:, j], fd0, atol=1e-8)
        assert np.allclose(B[:, j], fdb, atol=1e-8)


def _problem(seed=2, Ns=4):
    m = small()
    r = np.random.default_rng(seed)
    m0 = state(m, seed)
    dW = r.normal(scale=math.sqrt(m.dt), size=(Ns, m.K))
    lam = r.normal(scale=0.5, size=(Ns, m.K))
    _, u_end, _, _ = m.window(m0, dW, lam)
    y = u_end[:: m.n // 16][:16] + r.normal(scale=0.05, size=16)
    return m, m0, dW, lam, y


def test_gradient_matches_finite_differences_16_directions():
    m, m0, dW, lam, y = _problem()
    sigma = 0.05
    J, g = ON.cost_and_gradient(m, m0, dW, lam, y, sigma)
    assert np.isclose(J, ON.cost(m, m0, dW, lam, y, sigma), rtol=1e-14)
    r = np.random.default_rng(3)
    for _ in range(16):
        d = r.normal(size=lam.shape)
        eps = 1e-5
        fd = (ON.cost(m, m0, dW, lam + eps * d, y, sigma) - ON.cost(m, m0, dW, lam - eps * d, y, sigma)) / (2 * eps)
        assert abs(fd - np.sum(g * d)) <= 1e-6 * max(1.0, abs(fd))


def test_gradient_with_half_domain_observations():
    # Exp 2: observations on [0, L/2] only (y NaN elsewhere); the gradient still matches
    # central differences of the masked cost, and observations outside the mask do not matter
    m, m0, dW, lam, y = _problem()
    sigma = 0.05
    ym = y.copy()
    ym[len(y) // 2 + 1:] = np.nan
    J, g = ON.cost_and_gradient(m, m0, dW, lam, ym, sigma)
    assert np.isfinite(J) and np.all(np.isfinite(g))
    r = np.random.default_rng(4)
    for _ in range(4):
        d = r.normal(size=lam.shape)
        eps = 1e-5
        fd = (ON.cost(m, m0, dW, lam + eps * d, ym, sigma) - ON.cost(m, m0, dW, lam - eps * d, ym, sigma)) / (2 * eps)
        assert abs(fd - np.sum(g * d)) <= 1e-6 * max(1.0, abs(fd))
    # the terminal sensitivity vanishes at the unobserved nodes and is unchanged at the observed ones
    gm, gf = ON.obs_grad_u(m0, ym, sigma), ON.obs_grad_u(m0, y, sigma)
    stride = m.n // len(y)
    half = (len(y) // 2 + 1) * stride
    assert np.all(gm[half:] == 0.0) and np.array_equal(gm[:half], gf[:half])


def test_taylor_remainder_is_second_order():
    m, m0, dW, lam, y = _problem(4)
    sigma = 0.05
    J, g = ON.cost_and_gradient(m, m0, dW, lam, y, sigma)
    d = np.random.default_rng(5).normal(size=lam.shape)
    rem = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        rem.append(abs(ON.cost(m, m0, dW, lam + eps * d, y, sigma) - J - eps * np.sum(g * d)))
    assert 3.0 < rem[0] / rem[1] < 5.0 and 3.0 < rem[1] / rem[2] < 5.0


def test_open_loop_matches_linear_least_squares_in_linear_regime():
    m = small()
    Ns, K, sigma = 3, m.K, 0.05
    m0 = state(m, 6)
    zero = np.zeros((Ns, K))
    _, u_b, _, _ = m.window(m0, zero, zero)
    idx = OF.obs_indices(m.n, 16)
    dy = 1e-5 * np.random.default_rng(7).normal(size=16)
    y = u_b[idx] + dy
    # finite-difference Jacobian of the observed velocity with respect to lambda
    G = np.empty((16, Ns * K))
    eps = 1e-4
    for c in range(Ns * K):
        e = np.zeros(Ns * K)
        e[c] = eps
        up = m.window(m0, zero, e.reshape(Ns, K))[1][idx]
        um = m.window(m0, zero, -e.reshape(Ns, K))[1][idx]
        G[:, c] = (up - um) / (2 * eps)
    lam_ls = np.linalg.solve(G.T @ G / sigma ** 2 + m.dt * np.eye(Ns * K), G.T @ dy / sigma ** 2)
    lam_opt, res = ON.nudge_open_loop(m, m0, y, sigma, Ns, K, gtol=1e-14)
    assert np.max(np.abs(lam_opt.ravel() - lam_ls)) <= 1e-3 * np.max(np.abs(lam_ls)) + 1e-9


def test_sequential_schedule():
    m = small()
    Ns, K, sigma = 3, m.K, 0.05
    m0 = state(m, 8)
    _, u_b, _, _ = m.window(m0, np.zeros((Ns, K)))
    y = u_b[OF.obs_indices(m.n, 16)] + 0.05
    lam, dW = ON.nudge_sequential(m, m0, y, sigma, Ns, K, seed=3, particle=5, ctr=7)
    z = ORNG.normals(3, ORNG.TAG_NUDGE, K, np.arange(Ns, dtype=np.uint64), np.uint64(5), np.uint64(7))
    assert np.array_equal(dW, math.sqrt(m.dt) * z)
    # each stage ends at a stationary point of its own cost (later noise still zero)
    for n in range(Ns):
        dW_n = dW.copy()
        dW_n[n:] = 0.0
        lam_n = lam.copy()
        lam_n[n + 1:] = 0.0
        _, g = ON.cost_and_gradient(m, m0, dW_n, lam_n, y, sigma, var_steps=[n])
        assert np.max(np.abs(g)) < 1e-6
    # nudging lowers the misfit of the revealed path compared with no drift
    nll_nudged = OF.nll(m.window(m0, dW, lam)[1][None], y, sigma)[0]
    nll_plain = OF.nll(m.window(m0, dW)[1][None], y, sigma)[0]
    assert nll_nudged < nll_plain


def test_matern_gradient_matches_finite_differences():
    # the Matern noise (one Brownian motion per cell): the tangent-linear gradient over all
    # n drifts of every step against central differences of the cost, with a drift present,
    # and dJ/ddW = (dJ/dlambda - dt lambda) / dt (the noise depends on dW + lambda dt only)
    m = Model(L=40.0, n=64, alpha=1.0, mu=0.02, dt=0.025, amps=np.full(2, 0.05), noise_model="matern",
              kappa=1.0, eta=0.5, matern_k=3)
    r = np.random.default_rng(8)
    x = m.x
    u0 = 0.3 / np.cosh(x - 20.0) + 0.05 * np.sin(2 * math.pi * x / m.L)
    m0 = m.m_from_u(u0)
    Ns = 3
    dW = r.normal(scale=math.sqrt(m.dt), size=(Ns, m.n))
    lam = r.normal(scale=0.3, size=(Ns, m.n))
    y = u0[::4] + r.normal(scale=0.05, size=16)
    sigma = 0.05
    J, g = ON.cost_and_gradient(m, m0, dW, lam, y, sigma)
    assert g.shape == (Ns, m.n)
    assert np.isclose(J, ON.cost(m, m0, dW, lam, y, sigma), rtol=1e-14)
    for _ in range(8):
        d = r.normal(size=lam.shape)
        eps = 1e-5
        fd = (ON.cost(m, m0, dW, lam + eps * d, y, sigma) - ON.cost(m, m0, dW, lam - eps * d, y, sigma)) / (2 * eps)
        assert abs(fd - np.sum(g * d)) <= 1e-6 * max(1.0, abs(fd))
        fdw = (ON.cost(m, m0, dW + eps * d, lam, y, sigma) - ON.cost(m, m0, dW - eps * d, lam, y, sigma)) / (2 * eps)
        assert abs(fdw - np.sum((g - m.dt * lam) / m.dt * d)) <= 1e-6 * max(1.0, abs(fdw))
